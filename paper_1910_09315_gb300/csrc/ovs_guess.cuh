// Learned initial guess: per-grid network storage and launchers (see ovs_guess.cu).
#pragma once
#include <algorithm>

#include "ovs_internal.cuh"

namespace ovs {

// Per-grid region (inside the grid workspace), sized for the widest network (H = 128):
//   header | inference copy of the FP32 parameters | W2 as BF16 mma fragments | training: FP32 parameters,
//   Adam first and second moments, gradients, loss accumulator
struct MlpHeader {
    int32_t hidden;     // 0: no network
    int32_t ready;      // 1 once trained (or set) and packed
    float centre[3];    // input normalisation: xn = (x_body - centre) * inv_half
    float inv_half[3];
    int32_t pad[8];
};

struct GuessEntry {
    int32_t node;      // receiver node whose hint gets the guess
    int32_t receiver;  // receiver grid
    float x[3];        // normalised body-frame input
    int32_t pad;
};

// per donor grid, the start of its segment of the guess queue
struct GuessSeg {
    int64_t off[OVS_MAX_GRIDS];
};

constexpr int kMlpMaxHidden = 128;
constexpr int kMlpMaxParams = kMlpMaxHidden * kMlpMaxHidden + 8 * kMlpMaxHidden + 3;
constexpr size_t kMlpAlign(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kMlpFwOffset = 256;
constexpr size_t kMlpFragOffset = kMlpFwOffset + kMlpAlign(sizeof(float) * kMlpMaxParams);
constexpr size_t kMlpW3FragOffset = kMlpFragOffset + kMlpAlign(8 * (kMlpMaxHidden / 8) * (kMlpMaxHidden / 16) * 32);
constexpr size_t kMlpParamsOffset = kMlpW3FragOffset + kMlpAlign(8 * (kMlpMaxHidden / 16) * 32);
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
// always = 1: every point of a set whose first donor has a network gets its guess (hints ignored).
// counts: OVS_MAX_GRIDS counters (one per donor grid's segment of the queue).
cudaError_t launch_guess(const AsmParams& P, const GridDev* dgrids, int ngrids, const int* hidden, int always,
                         GuessEntry* queue, uint32_t* counts, int64_t cap, unsigned long long* used, cudaStream_t st);

}  // namespace ovs
