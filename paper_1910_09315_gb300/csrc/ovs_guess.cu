// Learned initial guess for the donor search of a body grid (not in the paper: the paper starts its walk from a
// control cell, Sec. 2.2.5).  A small network 3 -> H -> H -> 3 (SiLU) maps normalised body-frame coordinates to
// normalised curvilinear coordinates ((i + xi)/Ci, (j + eta)/Cj, (k + zeta)/Ck); the walk and the exact in-cell
// test then start from the cell it points at, so donors do not depend on the network.
//
//   k_train_samples  samples (cell, xi) -> network input (trilinear map of the cell, normalised) and target
//   k_train_grad     forward + backward of a mini-batch, one thread per sample, activations staged in shared
//                    memory, weight gradients reduced per block (FP32)
//   k_adam           Adam update of the FP32 parameters
//   k_pack           BF16 copy of the weights for inference, W2 in mma.sync fragment order
//   k_guess_select   points of a call that have no usable hint and a donor grid with a trained network ->
//                    compact queue of normalised body-frame inputs (warp ballot)
//   k_guess_mma      the network in BF16 on tensor cores (mma.sync m16n8k16, FP32 accumulation), 16 points per
//                    warp; writes the guessed cell into the receiver node's hint
//
// Parameter layout (FP32): W1 [H x 3] row-major, b1 [H], W2 [H x H] row-major (W2[out][in]), b2 [H], W3 [3 x H],
// b3 [3]: H*H + 8*H + 3 values.
#include <cuda_bf16.h>

#include "ovs_guess.cuh"

namespace ovs {

namespace {

__device__ __forceinline__ float silu(float z) { return z / (1.f + expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    float s = 1.f / (1.f + expf(-z));
    return s * (1.f + z * (1.f - s));
}

// ---------------------------------------------------------------------------------------------- samples
__global__ void k_train_samples(GridDev g, MlpHeader h, const int32_t* __restrict__ cells, const float* __restrict__ xi,
                                int64_t n, float* __restrict__ X, float* __restrict__ T) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t cell = cells[q];
        if (cell < 0 || cell >= g.ncells) cell = 0;
        double u = xi[q], v = xi[n + q], w = xi[2 * n + q];
        int i, j, k;
        cell_ijk(g, cell, i, j, k);
        double p[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            double wa = ((a & 1) ? u : 1 - u) * ((a & 2) ? v : 1 - v) * ((a & 4) ? w : 1 - w);
            int64_t nd = corner_node(g, i, j, k, a);
            p[0] += wa * g.x[nd];
            p[1] += wa * g.y[nd];
            p[2] += wa * g.z[nd];
        }
        double I[3] = {i + u, j + v, k + w};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            X[c * n + q] = (float)((p[c] - (double)h.centre[c]) * (double)h.inv_half[c]);
            T[c * n + q] = (float)(I[c] / (double)g.C[c]);
        }
    }
}

// ---------------------------------------------------------------------------------------------- training
template <int H>
struct TrainCfg {
    static constexpr int S = H >= 128 ? 64 : 128;  // samples per block
    static constexpr int NP = H * H + 8 * H + 3;
    static constexpr int HP = H + 1;  // padded row of the activation stages (no shared-memory bank conflicts)
    static constexpr size_t smem = sizeof(float) * (NP + (size_t)S * (4 * HP + 6));
};

template <int H>
__global__ void __launch_bounds__(TrainCfg<H>::S) k_train_grad(const float* __restrict__ params,
                                                               const float* __restrict__ X,
                                                               const float* __restrict__ T, int64_t n, int64_t off,
                                                               int64_t B, float inv_count, float* __restrict__ grads,
                                                               float* __restrict__ loss) {
    constexpr int S = TrainCfg<H>::S, NP = TrainCfg<H>::NP, HP = TrainCfg<H>::HP;
    extern __shared__ float sm[];
    float* W1 = sm;
    float* b1 = W1 + 3 * H;
    float* W2 = b1 + H;
    float* b2 = W2 + H * H;
    float* W3 = b2 + H;
    float* b3 = W3 + 3 * H;
    float* xs = sm + NP;     // [S][3]
    float* h1s = xs + 3 * S;    // [S][HP]
    float* a1s = h1s + S * HP;  // z1, then gz1
    float* h2s = a1s + S * HP;
    float* a2s = h2s + S * HP;  // z2, then gz2
    float* gys = a2s + S * HP;  // [S][3]
    for (int q = threadIdx.x; q < NP; q += S) sm[q] = params[q];
    __syncthreads();
    const int s = threadIdx.x;
    const int64_t q = off + (int64_t)blockIdx.x * S + s;
    const bool active = (int64_t)blockIdx.x * S + s < B && q < n;
    float x[3] = {0, 0, 0}, t[3] = {0, 0, 0};
    if (active) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            x[c] = X[c * n + q];
            t[c] = T[c * n + q];
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) xs[s * 3 + c] = x[c];
    // forward
    for (int j = 0; j < H; ++j) {
        float z = b1[j] + W1[3 * j] * x[0] + W1[3 * j + 1] * x[1] + W1[3 * j + 2] * x[2];
        a1s[s * HP + j] = z;
        h1s[s * HP + j] = silu(z);
    }
    for (int j = 0; j < H; ++j) {
        float z = b2[j];
        for (int k = 0; k < H; ++k) z += W2[j * H + k] * h1s[s * HP + k];
        a2s[s * HP + j] = z;
        h2s[s * HP + j] = silu(z);
    }
    float gy[3];
    float l = 0.f;
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        float y = b3[o];
        for (int k = 0; k < H; ++k) y += W3[o * H + k] * h2s[s * HP + k];
        float r = active ? y - t[o] : 0.f;
        l += r * r;
        gy[o] = 2.f * r * inv_count;
        gys[s * 3 + o] = gy[o];
    }
    // backward through the activations
    for (int k = 0; k < H; ++k) {
        float gh = W3[k] * gy[0] + W3[H + k] * gy[1] + W3[2 * H + k] * gy[2];
        a2s[s * HP + k] = gh * dsilu(a2s[s * HP + k]);  // gz2
    }
    for (int k = 0; k < H; ++k) {
        float gh = 0.f;
        for (int j = 0; j < H; ++j) gh += W2[j * H + k] * a2s[s * HP + j];
        a1s[s * HP + k] = gh * dsilu(a1s[s * HP + k]);  // gz1
    }
    // loss (sum of squares over the block)
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l * inv_count);
    __syncthreads();
    // weight gradients: block partial sums over its samples, one atomic per parameter and block
    for (int p = threadIdx.x; p < NP; p += S) {
        float acc = 0.f;
        if (p < 3 * H) {  // W1[j][c]
            int j = p / 3, c = p % 3;
            for (int r = 0; r < S; ++r) acc += a1s[r * HP + j] * xs[r * 3 + c];
        } else if (p < 4 * H) {  // b1
            int j = p - 3 * H;
            for (int r = 0; r < S; ++r) acc += a1s[r * HP + j];
        } else if (p < 4 * H + H * H) {  // W2[j][k]
            int jk = p - 4 * H, j = jk / H, k = jk % H;
            for (int r = 0; r < S; ++r) acc += a2s[r * HP + j] * h1s[r * HP + k];
        } else if (p < 5 * H + H * H) {  // b2
            int j = p - 4 * H - H * H;
            for (int r = 0; r < S; ++r) acc += a2s[r * HP + j];
        } else if (p < 8 * H + H * H) {  // W3[o][k]
            int ok = p - 5 * H - H * H, o = ok / H, k = ok % H;
            for (int r = 0; r < S; ++r) acc += gys[r * 3 + o] * h2s[r * HP + k];
        } else {  // b3
            int o = p - 8 * H - H * H;
            for (int r = 0; r < S; ++r) acc += gys[r * 3 + o];
        }
        if (acc != 0.f) atomicAdd(grads + p, acc);
    }
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int np, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < np; q += gridDim.x * blockDim.x) {
        float gq = g[q];
        float mq = b1 * m[q] + (1.f - b1) * gq;
        float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
        g[q] = 0.f;
    }
}

// ---------------------------------------------------------------------------------------------- inference
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// W2 fragments for mma.m16n8k16 with B[k][n] = W2[n][k]: per (n-tile, k-step, lane) two 32-bit registers:
// b0 = rows k = 2t, 2t+1; b1 = rows k = 2t+8, 2t+9 (t = lane % 4), column n = lane / 4.
__global__ void k_pack(const float* __restrict__ params, int H, float* __restrict__ fw, uint2* __restrict__ w2frag) {
    const int NP = H * H + 8 * H + 3;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NP; q += gridDim.x * blockDim.x) fw[q] = params[q];
    const float* W2 = params + 4 * H;
    const int nt = H / 8, ks = H / 16;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt * ks * 32; q += gridDim.x * blockDim.x) {
        int lane = q % 32, kk = (q / 32) % ks, n8 = q / (32 * ks);
        int g = lane >> 2, t = lane & 3;
        int n = 8 * n8 + g, k0 = 16 * kk + 2 * t;
        w2frag[q] = make_uint2(pack_bf16(W2[n * H + k0], W2[n * H + k0 + 1]),
                               pack_bf16(W2[n * H + k0 + 8], W2[n * H + k0 + 9]));
    }
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint2 b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// The network on 16 inputs held by one warp (row r of the tile: inputs xr[0..2] are read by the lanes that need
// them from `xin`, rows >= rows_valid are zero); returns y for rows g and g+8 in lanes with t == 0.
template <int H>
__device__ __forceinline__ void mlp_tile(const MlpHeader& hd, const float* __restrict__ fw,
                                         const uint2* __restrict__ w2frag, const float xin[16][3], float y[2][3]) {
    const int lane = (int)lane_id(), g = lane >> 2, t = lane & 3;
    const float* W1 = fw;
    const float* b1 = W1 + 3 * H;
    const float* b2 = b1 + H + H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + 3 * H;
    constexpr int KS = H / 16, NT = H / 8;
    // layer 1 straight into A fragments (rows g, g+8; columns 16kk + 2t + {0,1,8,9}), SiLU, BF16
    uint32_t A[KS][4];
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
        float h[2][4];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const float* xr = xin[g + 8 * rr];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int col = 16 * kk + 2 * t + (e & 1) + (e >> 1) * 8;
                float z = __ldg(b1 + col) + __ldg(W1 + 3 * col) * xr[0] + __ldg(W1 + 3 * col + 1) * xr[1] +
                          __ldg(W1 + 3 * col + 2) * xr[2];
                h[rr][e] = z / (1.f + __expf(-z));
            }
        }
        A[kk][0] = pack_bf16(h[0][0], h[0][1]);
        A[kk][1] = pack_bf16(h[1][0], h[1][1]);
        A[kk][2] = pack_bf16(h[0][2], h[0][3]);
        A[kk][3] = pack_bf16(h[1][2], h[1][3]);
    }
    // layer 2 on tensor cores, then SiLU and layer 3 partial sums over this lane's columns
    float part[2][3] = {{0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int n8 = 0; n8 < NT; ++n8) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < KS; ++kk) mma_bf16(c, A[kk], __ldg(w2frag + (n8 * KS + kk) * 32 + lane));
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int col = 8 * n8 + 2 * t + (e & 1);
            float z = c[e] + __ldg(b2 + col);
            float h2 = z / (1.f + __expf(-z));
            int rr = e >> 1;
#pragma unroll
            for (int o = 0; o < 3; ++o) part[rr][o] += __ldg(W3 + o * H + col) * h2;
        }
    }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            float v = part[rr][o];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            y[rr][o] = v + __ldg(b3 + o);
        }
}

// network evaluation on arbitrary inputs (normalised), for tests and direct use
template <int H>
__global__ void __launch_bounds__(128) k_guess_eval(MlpHeader hd, const float* __restrict__ fw,
                                                    const uint2* __restrict__ w2frag, const float* __restrict__ xn,
                                                    int64_t n, float* __restrict__ out) {
    __shared__ float xs[4][16][3];
    const int w = threadIdx.x >> 5, lane = (int)lane_id();
    const int64_t tiles = (n + 15) / 16;
    for (int64_t tile = blockIdx.x * 4 + w; tile < tiles; tile += (int64_t)gridDim.x * 4) {
        if (lane < 16) {
            int64_t q = tile * 16 + lane;
#pragma unroll
            for (int c = 0; c < 3; ++c) xs[w][lane][c] = q < n ? xn[c * n + q] : 0.f;
        }
        __syncwarp();
        float y[2][3];
        mlp_tile<H>(hd, fw, w2frag, xs[w], y);
        if ((lane & 3) == 0) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                int64_t q = tile * 16 + (lane >> 2) + 8 * rr;
                if (q < n)
#pragma unroll
                    for (int c = 0; c < 3; ++c) out[c * n + q] = y[rr][c];
            }
        }
        __syncwarp();
    }
}

// points without a usable hint whose first donor has a trained network -> guess queue
__global__ void __launch_bounds__(256) k_guess_select(const __grid_constant__ AsmParams P,
                                                      const GridDev* __restrict__ G, GuessEntry* __restrict__ queue,
                                                      uint32_t* __restrict__ count, int64_t cap, int always) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool want = false;
    GuessEntry e;
    if (t < P.total) {
        const int si = find_set(P.s, P.nsets, t);
        const SetDev& s = P.s[si];
        const int gd = s.donors[0];
        const GridDev& g = G[gd];
        const MlpHeader* hd = (const MlpHeader*)g.mlp;
        if (hd && hd->ready) {
            const int32_t node = __ldg(s.node_ids + (t - s.begin));
            const GridDev& gr = G[s.receiver];
            if (node >= 0 && node < gr.nnodes) {
                uint32_t h = gr.hint[node];
                bool valid = !always && h != kNoHint && (int)(h >> kCellBits) == gd &&
                             (h & ((1u << kCellBits) - 1)) < g.ncells;
                if (!valid) {
                    const int64_t nn = gr.nnodes;
                    ff x[3], xd[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        x[c] = {__ldg(gr.xff + 2 * c * nn + node), __ldg(gr.xff + (2 * c + 1) * nn + node)};
                    xf_apply(P.xf[si], x, xd);
                    bool inside = true;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float v = __fadd_rn(xd[c].hi, xd[c].lo);
                        inside = inside && v >= (float)g.lo[c] && v <= (float)g.hi[c];
                        e.x[c] = (v - hd->centre[c]) * hd->inv_half[c];
                    }
                    e.t = (int32_t)t;
                    want = inside;
                }
            }
        }
    }
    unsigned mask = __ballot_sync(0xffffffffu, want);
    if (mask) {
        const unsigned lane = lane_id();
        int leader = __ffs(mask) - 1;
        uint32_t base = 0;
        if ((int)lane == leader) base = atomicAdd(count, (uint32_t)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (want) {
            uint32_t idx = base + __popc(mask & ((1u << lane) - 1u));
            if (idx < cap) queue[idx] = e;
        }
    }
}

// guess queue -> hints (the network's cell), 16 points per warp
template <int H>
__global__ void __launch_bounds__(128) k_guess_mma(const __grid_constant__ AsmParams P, const GridDev* __restrict__ G,
                                                   const GuessEntry* __restrict__ queue,
                                                   const uint32_t* __restrict__ count, int64_t cap, int gd,
                                                   unsigned long long* __restrict__ used) {
    __shared__ float xs[4][16][3];
    __shared__ int32_t ts[4][16];
    const GridDev& g = G[gd];
    const MlpHeader hd = *(const MlpHeader*)g.mlp;
    const float* fw = (const float*)((const char*)g.mlp + kMlpFwOffset);
    const uint2* w2frag = (const uint2*)((const char*)g.mlp + kMlpFragOffset);
    const int w = threadIdx.x >> 5, lane = (int)lane_id();
    const int64_t n = min((int64_t)*count, cap);
    const int64_t tiles = (n + 15) / 16;
    unsigned nused = 0;
    for (int64_t tile = blockIdx.x * 4 + w; tile < tiles; tile += (int64_t)gridDim.x * 4) {
        if (lane < 16) {
            int64_t q = tile * 16 + lane;
            bool ok = false;
            if (q < n) {
                const GuessEntry e = queue[q];
                const int si = find_set(P.s, P.nsets, e.t);
                ok = P.s[si].donors[0] == gd;  // this launch handles donor grid gd
                ts[w][lane] = ok ? e.t : -1;
#pragma unroll
                for (int c = 0; c < 3; ++c) xs[w][lane][c] = ok ? e.x[c] : 0.f;
            } else {
                ts[w][lane] = -1;
#pragma unroll
                for (int c = 0; c < 3; ++c) xs[w][lane][c] = 0.f;
            }
        }
        __syncwarp();
        float y[2][3];
        mlp_tile<H>(hd, fw, w2frag, xs[w], y);
        if ((lane & 3) == 0) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int row = (lane >> 2) + 8 * rr;
                const int32_t t = ts[w][row];
                if (t < 0) continue;
                int ijk[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float I = y[rr][c] * (float)g.C[c];
                    int ci = (int)floorf(fminf(fmaxf(I, -1e6f), 1e6f));
                    if (g.per[c]) {
                        ci %= g.C[c];
                        if (ci < 0) ci += g.C[c];
                    } else {
                        ci = min(max(ci, 0), g.C[c] - 1);
                    }
                    ijk[c] = ci;
                }
                const int si = find_set(P.s, P.nsets, t);
                const SetDev& s = P.s[si];
                const int32_t node = __ldg(s.node_ids + (t - s.begin));
                G[s.receiver].hint[node] = ((uint32_t)gd << kCellBits) | (uint32_t)cell_id(g, ijk[0], ijk[1], ijk[2]);
                ++nused;
            }
        }
        __syncwarp();
    }
    if (used && nused) atomicAdd(used, (unsigned long long)nused);
}

}  // namespace

size_t mlp_region_bytes() { return kMlpRegionBytes; }

cudaError_t launch_train_samples(const GridDev& g, const MlpHeader& h, const int32_t* cells, const float* xi, int64_t n,
                                 float* X, float* T, cudaStream_t st) {
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_train_samples<<<blocks, 256, 0, st>>>(g, h, cells, xi, n, X, T);
    return cudaGetLastError();
}

template <int H>
static cudaError_t train_grad_h(const float* params, const float* X, const float* T, int64_t n, int64_t off, int64_t B,
                                float* grads, float* loss, float inv_count, cudaStream_t st) {
    using C = TrainCfg<H>;
    cudaError_t e = cudaFuncSetAttribute(k_train_grad<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (B + C::S - 1) / C::S;
    k_train_grad<H><<<(unsigned)blocks, C::S, C::smem, st>>>(params, X, T, n, off, B, inv_count, grads, loss);
    return cudaGetLastError();
}

cudaError_t launch_train_grad(int H, const float* params, const float* X, const float* T, int64_t n, int64_t off,
                              int64_t B, float* grads, float* loss, float inv_count, cudaStream_t st) {
    switch (H) {
        case 32: return train_grad_h<32>(params, X, T, n, off, B, grads, loss, inv_count, st);
        case 64: return train_grad_h<64>(params, X, T, n, off, B, grads, loss, inv_count, st);
        case 128: return train_grad_h<128>(params, X, T, n, off, B, grads, loss, inv_count, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adam(float* p, float* g, float* m, float* v, int np, float lr, int step, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(np + 255) / 256, 256, 0, st>>>(p, g, m, v, np, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float* params, int H, void* region, cudaStream_t st) {
    float* fw = (float*)((char*)region + kMlpFwOffset);
    uint2* w2 = (uint2*)((char*)region + kMlpFragOffset);
    k_pack<<<64, 256, 0, st>>>(params, H, fw, w2);
    return cudaGetLastError();
}

cudaError_t launch_guess_eval(int H, const void* region, const float* xn, int64_t n, float* out, cudaStream_t st) {
    MlpHeader hd = {};
    const float* fw = (const float*)((const char*)region + kMlpFwOffset);
    const uint2* w2 = (const uint2*)((const char*)region + kMlpFragOffset);
    int64_t tiles = (n + 15) / 16;
    unsigned blocks = (unsigned)std::min<int64_t>((tiles + 3) / 4, 152 * 8);
    if (blocks == 0) return cudaSuccess;
    switch (H) {
        case 32: k_guess_eval<32><<<blocks, 128, 0, st>>>(hd, fw, w2, xn, n, out); break;
        case 64: k_guess_eval<64><<<blocks, 128, 0, st>>>(hd, fw, w2, xn, n, out); break;
        case 128: k_guess_eval<128><<<blocks, 128, 0, st>>>(hd, fw, w2, xn, n, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_guess(const AsmParams& P, const GridDev* dgrids, int ngrids, const int* hidden, int always,
                         GuessEntry* queue, uint32_t* count, int64_t cap, unsigned long long* used, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    int64_t blocks = (P.total + 255) / 256;
    k_guess_select<<<(unsigned)blocks, 256, 0, st>>>(P, dgrids, queue, count, cap, always);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // one launch per donor grid with a network (the queue holds the points of all of them)
    unsigned gblocks = (unsigned)std::min<int64_t>((P.total / 16 + 3) / 4 + 1, 152 * 8);
    for (int gd = 0; gd < ngrids; ++gd) {
        if (hidden[gd] <= 0) continue;
        bool listed = false;
        for (int s = 0; s < P.nsets; ++s) listed = listed || P.s[s].donors[0] == gd;
        if (!listed) continue;
        switch (hidden[gd]) {
            case 32: k_guess_mma<32><<<gblocks, 128, 0, st>>>(P, dgrids, queue, count, cap, gd, used); break;
            case 64: k_guess_mma<64><<<gblocks, 128, 0, st>>>(P, dgrids, queue, count, cap, gd, used); break;
            case 128: k_guess_mma<128><<<gblocks, 128, 0, st>>>(P, dgrids, queue, count, cap, gd, used); break;
            default: break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ovs
