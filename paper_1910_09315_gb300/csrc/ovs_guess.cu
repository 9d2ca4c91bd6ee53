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

// B fragments for mma.m16n8k16 (B[k][n], k = 2t, 2t+1 in b0 and 2t+8, 2t+9 in b1, n = lane / 4, t = lane % 4):
//   layer 2: B[k][n] = W2[n][k], per (n-tile, k-step, lane);  layer 3: B[k][n] = W3[n][k] for n < 3, else 0.
__global__ void k_pack(const float* __restrict__ params, int H, float* __restrict__ fw, uint2* __restrict__ w2frag,
                       uint2* __restrict__ w3frag) {
    const int NP = H * H + 8 * H + 3;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NP; q += gridDim.x * blockDim.x) fw[q] = params[q];
    const float* W2 = params + 4 * H;
    const float* W3 = params + 5 * H + H * H;
    const int nt = H / 8, ks = H / 16;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt * ks * 32; q += gridDim.x * blockDim.x) {
        int lane = q % 32, kk = (q / 32) % ks, n8 = q / (32 * ks);
        int g = lane >> 2, t = lane & 3;
        int n = 8 * n8 + g, k0 = 16 * kk + 2 * t;
        w2frag[q] = make_uint2(pack_bf16(W2[n * H + k0], W2[n * H + k0 + 1]),
                               pack_bf16(W2[n * H + k0 + 8], W2[n * H + k0 + 9]));
    }
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < ks * 32; q += gridDim.x * blockDim.x) {
        int lane = q % 32, kk = q / 32;
        int g = lane >> 2, t = lane & 3, k0 = 16 * kk + 2 * t;
        float w[4] = {0.f, 0.f, 0.f, 0.f};
        if (g < 3) {
            w[0] = W3[g * H + k0];
            w[1] = W3[g * H + k0 + 1];
            w[2] = W3[g * H + k0 + 8];
            w[3] = W3[g * H + k0 + 9];
        }
        w3frag[q] = make_uint2(pack_bf16(w[0], w[1]), pack_bf16(w[2], w[3]));
    }
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint2 b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// One grid's network, staged in shared memory by a block
template <int H>
struct MlpSmem {
    float W1[3 * H];
    float b1[H];
    float b2[H];
    float W3[3 * H];
    float b3[4];
    uint2 w2[(H / 8) * (H / 16) * 32];
};

template <int H>
__device__ __forceinline__ void stage_mlp(MlpSmem<H>& S, const void* region) {
    const float* fw = (const float*)((const char*)region + kMlpFwOffset);
    const uint2* w2 = (const uint2*)((const char*)region + kMlpFragOffset);
    for (int q = threadIdx.x; q < 3 * H; q += blockDim.x) {
        S.W1[q] = fw[q];
        S.W3[q] = fw[5 * H + H * H + q];
    }
    for (int q = threadIdx.x; q < H; q += blockDim.x) {
        S.b1[q] = fw[3 * H + q];
        S.b2[q] = fw[4 * H + H * H + q];
    }
    if (threadIdx.x < 3) S.b3[threadIdx.x] = fw[8 * H + H * H + threadIdx.x];
    for (int q = threadIdx.x; q < (H / 8) * (H / 16) * 32; q += blockDim.x) S.w2[q] = w2[q];
}

// The network on a tile of 16 inputs (xin, one row per point) held by one warp.  Layer 1 in FP32 straight into
// the A fragments of layer 2; layer 2 on tensor cores (BF16 operands, FP32 accumulation); layer 3 in FP32 from
// the accumulator fragments, reduced over the 4 lanes of a row group.  On return, lanes with t = lane % 4 == 0
// hold y for rows g and g + 8 (g = lane / 4).
template <int H>
__device__ __forceinline__ void mlp_tile(const MlpSmem<H>& S, const float (*xin)[3], float y[2][3]) {
    const int lane = (int)lane_id(), g = lane >> 2, t = lane & 3;
    constexpr int KS = H / 16, NT = H / 8;
    float xr[2][3];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int c = 0; c < 3; ++c) xr[rr][c] = xin[g + 8 * rr][c];
    uint32_t A[KS][4];
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
        float h[2][4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int col = 16 * kk + 2 * t + (e & 1) + (e >> 1) * 8;
            const float w0 = S.W1[3 * col], w1 = S.W1[3 * col + 1], w2 = S.W1[3 * col + 2], bb = S.b1[col];
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                float z = bb + w0 * xr[rr][0] + w1 * xr[rr][1] + w2 * xr[rr][2];
                h[rr][e] = z / (1.f + __expf(-z));
            }
        }
        A[kk][0] = pack_bf16(h[0][0], h[0][1]);
        A[kk][1] = pack_bf16(h[1][0], h[1][1]);
        A[kk][2] = pack_bf16(h[0][2], h[0][3]);
        A[kk][3] = pack_bf16(h[1][2], h[1][3]);
    }
    // layer 2 on tensor cores; SiLU and the 64 -> 3 output layer in FP32 (its weights are large and its terms
    // cancel, so BF16 operands there would cost the guess its accuracy)
    float part[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int n8 = 0; n8 < NT; ++n8) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < KS; ++kk) mma_bf16(c, A[kk], S.w2[(n8 * KS + kk) * 32 + lane]);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int col = 8 * n8 + 2 * t + (e & 1);
            float z = c[e] + S.b2[col];
            float h2 = z / (1.f + __expf(-z));
            const int rr = e >> 1;
#pragma unroll
            for (int o = 0; o < 3; ++o) part[rr][o] += S.W3[o * H + col] * h2;
        }
    }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            float v = part[rr][o];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            y[rr][o] = v + S.b3[o];
        }
}

// network evaluation on arbitrary normalised inputs (tests and direct use)
template <int H>
__global__ void __launch_bounds__(128) k_guess_eval(const void* __restrict__ region, const float* __restrict__ xn,
                                                    int64_t n, float* __restrict__ out) {
    __shared__ MlpSmem<H> S;
    __shared__ float xs[4][16][3];
    stage_mlp<H>(S, region);
    __syncthreads();
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
        mlp_tile<H>(S, xs[w], y);
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

// points without a usable hint whose first donor has a trained network -> that grid's segment of the queue
__global__ void __launch_bounds__(256) k_guess_select(const __grid_constant__ AsmParams P,
                                                      const GridDev* __restrict__ G, GuessEntry* __restrict__ queue,
                                                      uint32_t* __restrict__ counts, GuessSeg seg, int always) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool want = false;
    int gd = -1;
    GuessEntry e;
    if (t < P.total) {
        const int si = find_set(P.s, P.nsets, t);
        const SetDev& s = P.s[si];
        gd = s.donors[0];
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
                    e.node = node;
                    e.receiver = s.receiver;
                    e.pad = 0;
                    want = inside;
                }
            }
        }
    }
    // one atomic per (warp, donor grid)
    const unsigned lane = lane_id();
    const unsigned group = __match_any_sync(0xffffffffu, want ? gd : -1);
    const int leader = __ffs(group) - 1;
    uint32_t base = 0;
    if (want && (int)lane == leader) base = atomicAdd(counts + gd, (uint32_t)__popc(group));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) queue[seg.off[gd] + base + __popc(group & ((1u << lane) - 1u))] = e;
}

// one donor grid's segment of the queue -> hints (the network's cell), 16 points per warp
template <int H>
__global__ void __launch_bounds__(128) k_guess_mma(const GridDev* __restrict__ G, int gd,
                                                   const GuessEntry* __restrict__ queue, const uint32_t* __restrict__ count,
                                                   unsigned long long* __restrict__ used) {
    __shared__ MlpSmem<H> S;
    __shared__ float xs[4][16][3];
    __shared__ int32_t nodes[4][16], recs[4][16];
    const GridDev& g = G[gd];
    stage_mlp<H>(S, g.mlp);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = (int)lane_id();
    const int64_t n = *count;
    const int64_t tiles = (n + 15) / 16;
    unsigned nused = 0;
    for (int64_t tile = blockIdx.x * 4 + w; tile < tiles; tile += (int64_t)gridDim.x * 4) {
        if (lane < 16) {
            int64_t q = tile * 16 + lane;
            if (q < n) {
                const GuessEntry e = queue[q];
                nodes[w][lane] = e.node;
                recs[w][lane] = e.receiver;
#pragma unroll
                for (int c = 0; c < 3; ++c) xs[w][lane][c] = e.x[c];
            } else {
                nodes[w][lane] = -1;
#pragma unroll
                for (int c = 0; c < 3; ++c) xs[w][lane][c] = 0.f;
            }
        }
        __syncwarp();
        float y[2][3];
        mlp_tile<H>(S, xs[w], y);
        if ((lane & 3) == 0) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int row = (lane >> 2) + 8 * rr;
                const int32_t node = nodes[w][row];
                if (node < 0) continue;
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
                G[recs[w][row]].hint[node] = ((uint32_t)gd << kCellBits) | (uint32_t)cell_id(g, ijk[0], ijk[1], ijk[2]);
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
    uint2* w3 = (uint2*)((char*)region + kMlpW3FragOffset);
    k_pack<<<64, 256, 0, st>>>(params, H, fw, w2, w3);
    return cudaGetLastError();
}

cudaError_t launch_guess_eval(int H, const void* region, const float* xn, int64_t n, float* out, cudaStream_t st) {
    int64_t tiles = (n + 15) / 16;
    unsigned blocks = (unsigned)std::min<int64_t>((tiles + 3) / 4, 152 * 8);
    if (blocks == 0) return cudaSuccess;
    switch (H) {
        case 32: k_guess_eval<32><<<blocks, 128, 0, st>>>(region, xn, n, out); break;
        case 64: k_guess_eval<64><<<blocks, 128, 0, st>>>(region, xn, n, out); break;
        case 128: k_guess_eval<128><<<blocks, 128, 0, st>>>(region, xn, n, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_guess(const AsmParams& P, const GridDev* dgrids, int ngrids, const int* hidden, int always,
                         GuessEntry* queue, uint32_t* counts, int64_t cap, unsigned long long* used, cudaStream_t st) {
    // segment of each donor grid: the points of the sets whose first donor it is (host knows the set sizes)
    GuessSeg seg;
    int64_t size[OVS_MAX_GRIDS] = {};
    for (int s = 0; s < P.nsets; ++s)
        if (hidden[P.s[s].donors[0]] > 0) size[P.s[s].donors[0]] += P.s[s].n;
    int64_t off = 0;
    for (int gd = 0; gd < OVS_MAX_GRIDS; ++gd) {
        seg.off[gd] = off;
        off += size[gd];
    }
    if (off > cap) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * OVS_MAX_GRIDS, st);
    if (e != cudaSuccess) return e;
    int64_t blocks = (P.total + 255) / 256;
    k_guess_select<<<(unsigned)blocks, 256, 0, st>>>(P, dgrids, queue, counts, seg, always);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int gd = 0; gd < ngrids; ++gd) {
        if (hidden[gd] <= 0 || size[gd] == 0) continue;
        unsigned gb = (unsigned)std::min<int64_t>((size[gd] / 16 + 3) / 4 + 1, 152 * 8);
        const GuessEntry* q = queue + seg.off[gd];
        switch (hidden[gd]) {
            case 32: k_guess_mma<32><<<gb, 128, 0, st>>>(dgrids, gd, q, counts + gd, used); break;
            case 64: k_guess_mma<64><<<gb, 128, 0, st>>>(dgrids, gd, q, counts + gd, used); break;
            case 128: k_guess_mma<128><<<gb, 128, 0, st>>>(dgrids, gd, q, counts + gd, used); break;
            default: break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ovs
