// Learned initial guess: per-grid network storage and launchers (see ovs_guess.cu).
#pragma once
#include <algorithm>

#include "ovs_internal.cuh"

namespace ovs {

// Per-grid region (inside the grid workspace), sized for the widest network (H = 128):
//   header | inference copy of the FP32 parameters | FP16 mma fragments of the three layers | b2 as FP16 pairs |
//   training: FP32 parameters, Adam first and second moments, gradients, loss accumulator
struct MlpHeader {
    int32_t hidden;     // 0: no network
    int32_t ready;      // 1 once trained (or set) and packed
    float centre[3];    // input normalisation: xn = (x_body - centre) * inv_half
    float inv_half[3];
    int32_t pad[8];
};

constexpr int kMlpMaxHidden = 128;
constexpr int kMlpMaxParams = kMlpMaxHidden * kMlpMaxHidden + 8 * kMlpMaxHidden + 3;
constexpr size_t kMlpAlign(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kMlpFwOffset = 256;
// FP16 mma fragments for inference (k_pack): W2 (2 H^2 bytes), layer 1 (32 H bytes), layer 3 (16 H bytes)
constexpr size_t kMlpW2FragOffset = kMlpFwOffset + kMlpAlign(sizeof(float) * kMlpMaxParams);
constexpr size_t kMlpW1FragOffset = kMlpW2FragOffset + kMlpAlign(2 * kMlpMaxHidden * kMlpMaxHidden);
constexpr size_t kMlpW3FragOffset = kMlpW1FragOffset + kMlpAlign(32 * kMlpMaxHidden);
constexpr size_t kMlpB2hOffset = kMlpW3FragOffset + kMlpAlign(16 * kMlpMaxHidden);
constexpr size_t kMlpParamsOffset = kMlpB2hOffset + kMlpAlign(2 * kMlpMaxHidden);
constexpr size_t kMlpMOffset = kMlpParamsOffset + kMlpAlign(sizeof(float) * kMlpMaxParams);
constexpr size_t kMlpVOffset = kMlpMOffset + kMlpAlign(sizeof(float) * kMlpMaxParams);
constexpr size_t kMlpGOffset = kMlpVOffset + kMlpAlign(sizeof(float) * kMlpMaxParams);
constexpr size_t kMlpLossOffset = kMlpGOffset + kMlpAlign(sizeof(float) * kMlpMaxParams);
constexpr size_t kMlpRegionBytes = kMlpLossOffset + 256;

inline int mlp_param_count(int H) { return H * H + 8 * H + 3; }

size_t mlp_region_bytes();
cudaError_t launch_train_samples(const GridDev& g, const MlpHeader& h, const int32_t* cells, const float* xi, int64_t n,
                                 float* X, float* T, cudaStream_t st);
cudaError_t launch_train_grad(int H, const float* params, const float* X, const float* T, int64_t n, int64_t off,
                              int64_t B, float* grads, float* loss, float inv_count, cudaStream_t st);
cudaError_t launch_adam(float* p, float* g, float* m, float* v, int np, float lr, int step, cudaStream_t st);
cudaError_t launch_pack(const float* params, int H, void* region, cudaStream_t st);
cudaError_t launch_guess_eval(int H, const void* region, const float* xn, int64_t n, float* out, cudaStream_t st);

}  // namespace ovs
