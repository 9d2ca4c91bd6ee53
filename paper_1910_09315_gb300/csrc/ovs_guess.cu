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
//   k_guess          points of a call that have no usable hint and a donor grid with a trained network, gathered
//                    per chunk into 16-row tiles -> the network (all layers in FP16 on tensor cores, mma.sync
//                    m16n8k16, FP32 accumulation) -> the guessed cell becomes the receiver node's hint
//
// Parameter layout (FP32): W1 [H x 3] row-major, b1 [H], W2 [H x H] row-major (W2[out][in]), b2 [H], W3 [3 x H],
// b3 [3]: H*H + 8*H + 3 values.
#include <cuda_fp16.h>

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
// FP16 pair, low half = first argument
__device__ __forceinline__ uint32_t pack_f16(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

// B fragments for mma.m16n8k16 (B[k][n]: k = 2t, 2t+1 in b0 and 2t+8, 2t+9 in b1, n = 8 * tile + lane / 4,
// t = lane % 4), FP16:
//   layer 1, one k-step per n-tile: rows k = 2c W1hi[n][c], 2c+1 W1hi[n][c], 6 b1hi[n], 7 b1lo[n], 8+2c W1lo[n][c],
//     9+2c and 14-15 zero, against A = (x_hi c, x_lo c) in columns 2c, 2c+1, ones in 6-7, (x_hi c, 0) in 8+2c, 9+2c
//     (c = 0..2), so layer 1 keeps about FP32 accuracy and lane t of a row group needs component t only;
//   layer 2: W2[n][k], two consecutive k-steps per 16-byte entry, per (n-tile, k-step pair, lane), accumulated in
//     FP16 (its outputs feed the next FP16 operand directly);
//   layer 3, one n-tile: n = 0-2 W3hi[n][k], 3-5 W3lo[n - 3][k], 6-7 zero; output o is column o plus column o + 3.
__global__ void k_pack(const float* __restrict__ params, int H, float* __restrict__ fw, uint2* __restrict__ w1frag,
                       uint4* __restrict__ w2frag, uint2* __restrict__ w3frag) {
    const int NP = H * H + 8 * H + 3;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int q = tid; q < NP; q += nth) fw[q] = params[q];
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

__device__ __forceinline__ void mma_f16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint2 b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b.x), "r"(b.y));
}

// FP16 accumulators: d (rows g, g+8 as FP16 pairs) += A B
__device__ __forceinline__ void mma_f16_acc16(uint32_t d[2], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                              uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f16.f16.f16.f16 {%0,%1}, {%2,%3,%4,%5}, {%6,%7}, {%0,%1};\n"
                 : "+r"(d[0]), "+r"(d[1])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// SiLU of an FP16 pair: z * sigmoid(z) = z/2 * (1 + tanh(z/2)), one hardware tanh for both (its error, about
// 2^-11, is that of the FP16 rounding itself; the guess only picks the walk's start, donors do not depend on it)
__device__ __forceinline__ uint32_t silu_h2(uint32_t zb) {
    const __half2 h = __hmul2(*reinterpret_cast<const __half2*>(&zb), __float2half2_rn(0.5f));
    const uint32_t hb = *reinterpret_cast<const uint32_t*>(&h);
    uint32_t tb;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(tb) : "r"(hb));
    const __half2 r = __hfma2(h, *reinterpret_cast<const __half2*>(&tb), h);
    return *reinterpret_cast<const uint32_t*>(&r);
}

// One grid's network in shared memory: the FP16 fragments k_pack wrote, b2 as FP16 pairs (the layer-2
// accumulators start from it) and b3
template <int H>
struct MlpSmem {
    uint2 w1[(H / 8) * 32];
    uint4 w2[(H / 8) * (H / 32) * 32];
    uint2 w3[(H / 16) * 32];
    uint32_t b2[H / 2];
    float4 b3;
};

template <int H>
__device__ __forceinline__ void stage_mlp(MlpSmem<H>& S, const void* region) {
    const float* fw = (const float*)((const char*)region + kMlpFwOffset);
    const uint2* w1 = (const uint2*)((const char*)region + kMlpW1FragOffset);
    const uint4* w2 = (const uint4*)((const char*)region + kMlpW2FragOffset);
    const uint2* w3 = (const uint2*)((const char*)region + kMlpW3FragOffset);
    for (int q = threadIdx.x; q < (H / 8) * 32; q += blockDim.x) S.w1[q] = w1[q];
    for (int q = threadIdx.x; q < (H / 8) * (H / 32) * 32; q += blockDim.x) S.w2[q] = w2[q];
    for (int q = threadIdx.x; q < (H / 16) * 32; q += blockDim.x) S.w3[q] = w3[q];
    for (int q = threadIdx.x; q < H / 2; q += blockDim.x)
        S.b2[q] = pack_f16(fw[4 * H + H * H + 2 * q], fw[4 * H + H * H + 2 * q + 1]);
    if (threadIdx.x == 0) {
        const float* b3 = fw + 8 * H + H * H;
        S.b3 = make_float4(b3[0], b3[1], b3[2], 0.f);
    }
}

// The network on a tile of 16 inputs (xin[r].xyz, one row per point) held by one warp, all three layers on tensor
// cores (mma.sync m16n8k16, FP16 operands).  An m16n8 accumulator pair (n-tiles 2k, 2k + 1) has the layout of the
// m16k16 A operand of the next layer's k-step k, so activations stay in registers:
//   layer 1: x split into FP16 hi/lo against (W1hi, W1lo, b1hi, b1lo), FP32 accumulation -> z1 to ~FP32;
//   layer 2: SiLU(z1) in FP16 against W2 in FP16, FP16 accumulators starting from b2;
//   layer 3: SiLU(z2) in FP16 against W3 split into hi and lo columns, FP32 accumulation; y_o = column o +
//   column o + 3 + b3_o.
// On return, lanes with t = lane % 4 == 0 hold y for rows g and g + 8 (g = lane / 4).
template <int H>
__device__ __forceinline__ void mlp_tile(const MlpSmem<H>& S, const float4* xin, float y[2][3]) {
    const int lane = (int)lane_id(), g = lane >> 2, t = lane & 3;
    constexpr int KS = H / 16, NT = H / 8;
    // layer-1 A fragment (columns 2t, 2t+1 in a0 row g / a1 row g+8; 2t+8, 2t+9 in a2 / a3): component t's
    // (x_hi, x_lo) and (x_hi, 0) for t < 3, (1, 1) and (0, 0) for t = 3
    uint32_t a1f[4];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const float4 r = xin[g + 8 * rr];
        const float xt = t == 0 ? r.x : (t == 1 ? r.y : r.z);
        const float xh = __half2float(__float2half_rn(xt));
        const float xl = xt - xh;
        a1f[rr] = t == 3 ? pack_f16(1.f, 1.f) : pack_f16(xh, xl);
        a1f[2 + rr] = t == 3 ? 0u : pack_f16(xh, 0.f);
    }
    // layer 1 -> SiLU -> A fragments of layer 2
    uint32_t A[KS][4];
#pragma unroll
    for (int n8 = 0; n8 < NT; ++n8) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma_f16(c, a1f[0], a1f[1], a1f[2], a1f[3], S.w1[n8 * 32 + lane]);
        A[n8 >> 1][(n8 & 1) * 2] = silu_h2(pack_f16(c[0], c[1]));
        A[n8 >> 1][(n8 & 1) * 2 + 1] = silu_h2(pack_f16(c[2], c[3]));
    }
    // layer 2 -> SiLU -> layer 3: n-tiles 2k and 2k + 1 of layer 2 make the A fragment of layer 3's k-step k
    float c3[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
        uint32_t a3[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int n8 = 2 * kk + h;
            const uint32_t bb = S.b2[4 * n8 + t];
            uint32_t d[2] = {bb, bb};
#pragma unroll
            for (int kp = 0; kp < KS / 2; ++kp) {
                const uint4 b = S.w2[(n8 * (KS / 2) + kp) * 32 + lane];
                mma_f16_acc16(d, A[2 * kp][0], A[2 * kp][1], A[2 * kp][2], A[2 * kp][3], b.x, b.y);
                mma_f16_acc16(d, A[2 * kp + 1][0], A[2 * kp + 1][1], A[2 * kp + 1][2], A[2 * kp + 1][3], b.z, b.w);
            }
            a3[2 * h] = silu_h2(d[0]);
            a3[2 * h + 1] = silu_h2(d[1]);
        }
        mma_f16(c3, a3[0], a3[1], a3[2], a3[3], S.w3[kk * 32 + lane]);
    }
    // lane t holds columns 2t, 2t+1 of rows g (c3[0], c3[1]) and g+8 (c3[2], c3[3])
    float s1[4], s2[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        s1[e] = __shfl_down_sync(0xffffffffu, c3[e], 1);  // columns 2, 3
        s2[e] = __shfl_down_sync(0xffffffffu, c3[e], 2);  // columns 4, 5
    }
    const float4 b3 = S.b3;
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        y[rr][0] = c3[2 * rr] + s1[2 * rr + 1] + b3.x;
        y[rr][1] = c3[2 * rr + 1] + s2[2 * rr] + b3.y;
        y[rr][2] = s1[2 * rr] + s2[2 * rr + 1] + b3.z;
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

// Persistent blocks over the chunks of the sets that take a guess.  Per chunk, phase A (every thread, four points
// each, independent loads): the points without a usable hint whose position lies in the donor grid's box are
// gathered into shared memory (network input and receiver node); phase B (warps, 16 rows a tile): the network
// on the gathered rows, and the guessed cell becomes the receiver node's hint.  A block stages a network only
// when its chunk's donor grid changes.
template <int H>
__global__ void __launch_bounds__(128, kGuessBlocksPerSM) k_guess(const StepParams* __restrict__ Sp,
                                                                   const GridDev* __restrict__ G) {
    const AsmParams& P = Sp->a;
    const GuessWork& W = Sp->w[H == 32 ? 0 : (H == 64 ? 1 : 2)];
    const int always = P.guess_always;
    unsigned long long* __restrict__ used = P.guess_used;
    constexpr int kPer = kGuessChunk / 128;
    __shared__ MlpSmem<H> S;
    __shared__ float4 rows[kGuessChunk + 16];  // xyz = network input, w = receiver node (bits)
    __shared__ int nrows;
    __shared__ struct {
        float lo[3], hi[3], centre[3], inv_half[3], Cf[3], invC[3];
        int C[3], per[3];
    } K;  // the chunk's donor grid: box, input normalisation, cell counts
    const int wp = threadIdx.x >> 5, lane = (int)lane_id();
    const int64_t nchunks = W.chunk_begin[W.nsets];
    int staged = -1;
    unsigned nused = 0;
    for (int64_t chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        int w = 0;
        while (w + 1 < W.nsets && W.chunk_begin[w + 1] <= chunk) ++w;
        const int si = W.set[w];
        const SetDev& s = P.s[si];
        const int gd = s.donors[0];
        const GridDev& g = G[gd];
        const GridDev& gr = G[s.receiver];
        __syncthreads();  // the previous chunk's rows (and network) are no longer read
        if (gd != staged) {
            stage_mlp<H>(S, g.mlp);
            staged = gd;
        }
        if (threadIdx.x == 0) {
            nrows = 0;
            const MlpHeader* hd = (const MlpHeader*)g.mlp;
            for (int c = 0; c < 3; ++c) {
                K.lo[c] = (float)g.lo[c];
                K.hi[c] = (float)g.hi[c];
                K.centre[c] = hd->centre[c];
                K.inv_half[c] = hd->inv_half[c];
                K.Cf[c] = (float)g.C[c];
                K.invC[c] = 1.f / (float)g.C[c];
                K.C[c] = g.C[c];
                K.per[c] = g.per[c];
            }
        }
        __syncthreads();
        const int64_t nn = gr.nnodes;
        const uint32_t ncells = (uint32_t)g.ncells;
        uint32_t* __restrict__ hint = gr.hint;
        const int64_t c0 = (chunk - W.chunk_begin[w]) * kGuessChunk;
        const int64_t c1 = min(c0 + (int64_t)kGuessChunk, s.n);
        // phase A
        int32_t node[kPer];
        uint32_t h[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t q = c0 + 128 * k + threadIdx.x;
            node[k] = q < c1 ? __ldg(s.node_ids + q) : -1;
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) h[k] = (node[k] >= 0 && node[k] < nn) ? hint[node[k]] : 0u;
        const XfFF& xf = P.xf[si];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            bool want = false;
            float4 r;
            if (node[k] >= 0 && node[k] < nn) {
                const bool valid = !always && h[k] != kNoHint && (int)(h[k] >> kCellBits) == gd &&
                                   (h[k] & ((1u << kCellBits) - 1)) < ncells;
                if (!valid) {
                    // the network's input needs no more than FP32: the high parts of position and map
                    float x[3], v[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) x[c] = __ldg(gr.xff + 2 * c * nn + node[k]);
                    bool inside = true;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        v[c] = fmaf(xf.Mh[3 * c + 2], x[2],
                                    fmaf(xf.Mh[3 * c + 1], x[1], fmaf(xf.Mh[3 * c], x[0], xf.th[c])));
                        inside = inside && v[c] >= K.lo[c] && v[c] <= K.hi[c];
                        v[c] = (v[c] - K.centre[c]) * K.inv_half[c];
                    }
                    r = make_float4(v[0], v[1], v[2], __int_as_float(node[k]));
                    want = inside;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, want);
            int base = 0;
            if (lane == 0 && bal) base = atomicAdd(&nrows, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (want) rows[base + __popc(bal & ((1u << lane) - 1u))] = r;
        }
        __syncthreads();
        const int n = nrows;
        if ((int)threadIdx.x < ((n + 15) & ~15) - n) rows[n + threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        // phase B
        const int t = lane & 3, gq = lane >> 2;
        for (int t0 = 16 * wp; t0 < n; t0 += 64) {
            float y[2][3];
            mlp_tile<H>(S, rows + t0, y);
            // lane 4g keeps row g, lane 4g + 1 takes row g + 8
            float yr[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float o = __shfl_up_sync(0xffffffffu, y[1][c], 1);
                yr[c] = t == 0 ? y[0][c] : o;
            }
            const int row = t0 + gq + 8 * t;
            if (t < 2 && row < n) {
                int ijk[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float f = fminf(fmaxf(yr[c] * K.Cf[c], -1e6f), 1e6f);
                    if (K.per[c]) f -= K.Cf[c] * floorf(f * K.invC[c]);
                    ijk[c] = min(max((int)floorf(f), 0), K.C[c] - 1);
                }
                hint[__float_as_int(rows[row].w)] =
                    ((uint32_t)gd << kCellBits) | (uint32_t)(ijk[0] + K.C[0] * (ijk[1] + K.C[1] * ijk[2]));
                ++nused;
            }
        }
    }
    if (used) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, nused);
        if (lane == 0 && tot) atomicAdd(used, (unsigned long long)tot);
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
    k_pack<<<64, 256, 0, st>>>(params, H, fw, w1, w2, w3);
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

void fill_guess_work(const AsmParams& P, const int* hidden, GuessWork Wk[3]) {
    const int widths[3] = {32, 64, 128};
    for (int h = 0; h < 3; ++h) {
        GuessWork& W = Wk[h];
        W.nsets = 0;
        int64_t chunks = 0;
        for (int s = 0; s < P.nsets; ++s) {
            if (hidden[P.s[s].donors[0]] != widths[h] || P.s[s].n <= 0) continue;
            W.set[W.nsets] = s;
            W.chunk_begin[W.nsets] = chunks;
            chunks += (P.s[s].n + kGuessChunk - 1) / kGuessChunk;
            ++W.nsets;
        }
        W.chunk_begin[W.nsets] = chunks;
    }
}

cudaError_t launch_guess(const StepParams* dS, const GridDev* dgrids, int hmask, int nsm, int bps, cudaStream_t st) {
    // one persistent launch per network width present; its blocks walk that width's chunk list (possibly empty)
    const unsigned blocks = (unsigned)(nsm * (bps > 0 ? bps : kGuessBlocksPerSM));
    if (hmask & 1) k_guess<32><<<blocks, 128, 0, st>>>(dS, dgrids);
    if (hmask & 2) k_guess<64><<<blocks, 128, 0, st>>>(dS, dgrids);
    if (hmask & 4) k_guess<128><<<blocks, 128, 0, st>>>(dS, dgrids);
    return cudaGetLastError();
}

}  // namespace ovs
