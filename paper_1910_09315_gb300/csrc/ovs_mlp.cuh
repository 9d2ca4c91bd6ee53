// Inference of the learned-guess network 3 -> H -> H -> 3 (SiLU) on tensor cores, one 16-row tile per warp
// (mma.sync m16n8k16, FP16 operands).  Shared by the network evaluation kernel (weights staged in shared memory)
// and the assembly kernel (weights read from the grid's network region through the L1 cache).
#pragma once
#include <cuda_fp16.h>

#include "ovs_guess.cuh"

namespace ovs {

// FP16 pair, low half = first argument
__device__ __forceinline__ uint32_t pack_f16(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
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
    __device__ __forceinline__ uint2 W1(int q) const { return w1[q]; }
    __device__ __forceinline__ uint4 W2(int q) const { return w2[q]; }
    __device__ __forceinline__ uint2 W3(int q) const { return w3[q]; }
    __device__ __forceinline__ uint32_t B2(int q) const { return b2[q]; }
    __device__ __forceinline__ float4 B3() const { return b3; }
};

// The same network read in place from its region (the fragments are laid out per lane, so every read of a warp
// is one contiguous, coalesced span; repeated tiles hit the L1 cache).
template <int H>
struct MlpGlobal {
    const uint2* w1;
    const uint4* w2;
    const uint2* w3;
    const uint32_t* b2;
    const float* b3;
    __device__ __forceinline__ explicit MlpGlobal(const void* region)
        : w1((const uint2*)((const char*)region + kMlpW1FragOffset)),
          w2((const uint4*)((const char*)region + kMlpW2FragOffset)),
          w3((const uint2*)((const char*)region + kMlpW3FragOffset)),
          b2((const uint32_t*)((const char*)region + kMlpB2hOffset)),
          b3((const float*)((const char*)region + kMlpFwOffset) + 8 * H + H * H) {}
    __device__ __forceinline__ uint2 W1(int q) const { return __ldg(w1 + q); }
    __device__ __forceinline__ uint4 W2(int q) const { return __ldg(w2 + q); }
    __device__ __forceinline__ uint2 W3(int q) const { return __ldg(w3 + q); }
    __device__ __forceinline__ uint32_t B2(int q) const { return __ldg(b2 + q); }
    __device__ __forceinline__ float4 B3() const { return make_float4(__ldg(b3), __ldg(b3 + 1), __ldg(b3 + 2), 0.f); }
};

template <int H>
__device__ __forceinline__ void stage_mlp(MlpSmem<H>& S, const void* region) {
    const uint2* w1 = (const uint2*)((const char*)region + kMlpW1FragOffset);
    const uint4* w2 = (const uint4*)((const char*)region + kMlpW2FragOffset);
    const uint2* w3 = (const uint2*)((const char*)region + kMlpW3FragOffset);
    const uint32_t* b2 = (const uint32_t*)((const char*)region + kMlpB2hOffset);
    const float* fw = (const float*)((const char*)region + kMlpFwOffset);
    for (int q = threadIdx.x; q < (H / 8) * 32; q += blockDim.x) S.w1[q] = w1[q];
    for (int q = threadIdx.x; q < (H / 8) * (H / 32) * 32; q += blockDim.x) S.w2[q] = w2[q];
    for (int q = threadIdx.x; q < (H / 16) * 32; q += blockDim.x) S.w3[q] = w3[q];
    for (int q = threadIdx.x; q < H / 2; q += blockDim.x) S.b2[q] = b2[q];
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
// On return, lanes with t = lane % 4 == 0 hold y for rows g and g + 8 (g = lane / 4).  All 32 lanes call it.
template <int H, class Src>
__device__ __forceinline__ void mlp_tile(const Src& S, const float4* xin, float y[2][3]) {
    const int lane = (int)(threadIdx.x & 31u), g = lane >> 2, t = lane & 3;
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
        mma_f16(c, a1f[0], a1f[1], a1f[2], a1f[3], S.W1(n8 * 32 + lane));
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
            const uint32_t bb = S.B2(4 * n8 + t);
            uint32_t d[2] = {bb, bb};
#pragma unroll
            for (int kp = 0; kp < KS / 2; ++kp) {
                const uint4 b = S.W2((n8 * (KS / 2) + kp) * 32 + lane);
                mma_f16_acc16(d, A[2 * kp][0], A[2 * kp][1], A[2 * kp][2], A[2 * kp][3], b.x, b.y);
                mma_f16_acc16(d, A[2 * kp + 1][0], A[2 * kp + 1][1], A[2 * kp + 1][2], A[2 * kp + 1][3], b.z, b.w);
            }
            a3[2 * h] = silu_h2(d[0]);
            a3[2 * h + 1] = silu_h2(d[1]);
        }
        mma_f16(c3, a3[0], a3[1], a3[2], a3[3], S.W3(kk * 32 + lane));
    }
    // lane t holds columns 2t, 2t+1 of rows g (c3[0], c3[1]) and g+8 (c3[2], c3[3])
    float s1[4], s2[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        s1[e] = __shfl_down_sync(0xffffffffu, c3[e], 1);  // columns 2, 3
        s2[e] = __shfl_down_sync(0xffffffffu, c3[e], 2);  // columns 4, 5
    }
    const float4 b3 = S.B3();
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        y[rr][0] = c3[2 * rr] + s1[2 * rr + 1] + b3.x;
        y[rr][1] = c3[2 * rr + 1] + s2[2 * rr] + b3.y;
        y[rr][2] = s1[2 * rr] + s2[2 * rr + 1] + b3.z;
    }
}

}  // namespace ovs
