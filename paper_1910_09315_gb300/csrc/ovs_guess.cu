// Learned initial guess for the donor search of a body grid (not in the paper: the paper starts its walk from a
// control cell, Sec. 2.2.5).  A small network 3 -> H -> H -> 3 (SiLU) maps normalised body-frame coordinates to
// normalised curvilinear coordinates ((i + xi)/Ci, (j + eta)/Cj, (k + zeta)/Ck); the walk and the exact in-cell
// test then start from the cell it points at, so donors do not depend on the network.
//
//   k_train_samples  samples (cell, xi) -> network input (trilinear map of the cell, normalised) and target
//   k_train_grad     forward + backward of a mini-batch, one thread per sample, activations staged in shared
//                    memory, weight gradients reduced per block (FP32)
//   k_adam           Adam update of the FP32 parameters
//   k_pack           FP32 copy of the biases and FP16 mma.sync fragments of the three layers for inference
//   k_guess_eval     the network on given inputs (ovs_guess_eval; the same tile code, ovs_mlp.cuh, runs inside
//                    k_assemble for the points of a call that have no usable hint)
//
// Parameter layout (FP32): W1 [H x 3] row-major, b1 [H], W2 [H x H] row-major (W2[out][in]), b2 [H], W3 [3 x H],
// b3 [3]: H*H + 8*H + 3 values.
#include "ovs_mlp.cuh"

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

// B fragments for mma.m16n8k16 (B[k][n]: k = 2t, 2t+1 in b0 and 2t+8, 2t+9 in b1, n = 8 * tile + lane / 4,
// t = lane % 4), FP16:
//   layer 1, one k-step per n-tile: rows k = 2c W1hi[n][c], 2c+1 W1hi[n][c], 6 b1hi[n], 7 b1lo[n], 8+2c W1lo[n][c],
//     9+2c and 14-15 zero, against A = (x_hi c, x_lo c) in columns 2c, 2c+1, ones in 6-7, (x_hi c, 0) in 8+2c, 9+2c
//     (c = 0..2), so layer 1 keeps about FP32 accuracy and lane t of a row group needs component t only;
//   layer 2: W2[n][k], two consecutive k-steps per 16-byte entry, per (n-tile, k-step pair, lane), accumulated in
//     FP16 (its outputs feed the next FP16 operand directly);
//   layer 3, one n-tile: n = 0-2 W3hi[n][k], 3-5 W3lo[n - 3][k], 6-7 zero; output o is column o plus column o + 3.
// b2h: b2 as FP16 pairs (the initial values of the layer-2 FP16 accumulators).
__global__ void k_pack(const float* __restrict__ params, int H, float* __restrict__ fw, uint2* __restrict__ w1frag,
                       uint4* __restrict__ w2frag, uint2* __restrict__ w3frag, uint32_t* __restrict__ b2h) {
    const int NP = H * H + 8 * H + 3;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int q = tid; q < NP; q += nth) fw[q] = params[q];
    for (int q = tid; q < H / 2; q += nth) b2h[q] = pack_f16(params[4 * H + H * H + 2 * q], params[4 * H + H * H + 2 * q + 1]);
    const float* W1 = params;
    const float* b1 = params + 3 * H;
    const float* W2 = params + 4 * H;
    const float* W3 = params + 5 * H + H * H;
    const int nt = H / 8, kp = H / 32, ks = H / 16;
    auto hi = [](float v) { return __half2float(__float2half_rn(v)); };
    auto b1row = [&](int k, int n) -> float {
        if (k < 6) return hi(W1[3 * n + k / 2]);  // against x_hi (even k) and x_lo (odd k) of component k / 2
        if (k == 6) return hi(b1[n]);
        if (k == 7) return b1[n] - hi(b1[n]);
        if (k < 14 && k % 2 == 0) return W1[3 * n + (k - 8) / 2] - hi(W1[3 * n + (k - 8) / 2]);  // against x_hi
        return 0.f;
    };
    for (int q = tid; q < nt * 32; q += nth) {
        const int lane = q % 32, n = 8 * (q / 32) + lane / 4, t = lane % 4;
        w1frag[q] = make_uint2(pack_f16(b1row(2 * t, n), b1row(2 * t + 1, n)),
                               pack_f16(b1row(2 * t + 8, n), b1row(2 * t + 9, n)));
    }
    for (int q = tid; q < nt * kp * 32; q += nth) {
        const int lane = q % 32, pp = (q / 32) % kp, n8 = q / (32 * kp);
        const int n = 8 * n8 + lane / 4, t = lane % 4;
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k0 = 16 * (2 * pp + h) + 2 * t;
            w[2 * h] = pack_f16(W2[n * H + k0], W2[n * H + k0 + 1]);
            w[2 * h + 1] = pack_f16(W2[n * H + k0 + 8], W2[n * H + k0 + 9]);
        }
        w2frag[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    auto b3row = [&](int k, int n) -> float {
        if (n < 3) return hi(W3[n * H + k]);
        if (n < 6) return W3[(n - 3) * H + k] - hi(W3[(n - 3) * H + k]);
        return 0.f;
    };
    for (int q = tid; q < ks * 32; q += nth) {
        const int lane = q % 32, kk = q / 32, n = lane / 4, k0 = 16 * kk + 2 * (lane % 4);
        w3frag[q] = make_uint2(pack_f16(b3row(k0, n), b3row(k0 + 1, n)), pack_f16(b3row(k0 + 8, n), b3row(k0 + 9, n)));
    }
}

// network evaluation on arbitrary normalised inputs (tests and direct use)
template <int H>
__global__ void __launch_bounds__(128) k_guess_eval(const void* __restrict__ region, const float* __restrict__ xn,
                                                    int64_t n, float* __restrict__ out) {
    __shared__ MlpSmem<H> S;
    __shared__ float4 xs[4][16];
    stage_mlp<H>(S, region);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = (int)lane_id();
    const int64_t tiles = (n + 15) / 16;
    for (int64_t tile = blockIdx.x * 4 + w; tile < tiles; tile += (int64_t)gridDim.x * 4) {
        if (lane < 16) {
            int64_t q = tile * 16 + lane;
            xs[w][lane] = q < n ? make_float4(xn[q], xn[n + q], xn[2 * n + q], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
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
    uint2* w1 = (uint2*)((char*)region + kMlpW1FragOffset);
    uint4* w2 = (uint4*)((char*)region + kMlpW2FragOffset);
    uint2* w3 = (uint2*)((char*)region + kMlpW3FragOffset);
    uint32_t* b2h = (uint32_t*)((char*)region + kMlpB2hOffset);
    k_pack<<<64, 256, 0, st>>>(params, H, fw, w1, w2, w3, b2h);
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

}  // namespace ovs
