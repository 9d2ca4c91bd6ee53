// Contravariant fluxes at the receivers and the mass-conservation correction (see ovs_flux.cu).
#pragma once
#include <algorithm>

#include "ovs_internal.cuh"

namespace ovs {

constexpr int kMaxFluxSurfaces = 64;

struct FluxParams {
    int32_t grid;
    int32_t nsurf;
    int64_t nfaces;
    const int64_t* faces;  // face id = 3 * base node + d
    const int8_t* signs;   // +1 / -1 per face (NULL: all +1)
    FieldsDev vel;         // node velocities u, v, w of the grid
    void* flux;            // [nfaces], the fields' type
    double* net;           // [2 nsurf]: net signed flux before the correction, total face area
    int32_t* err;
    int32_t pad;
    int64_t surf_start[kMaxFluxSurfaces + 1];
};

cudaError_t launch_flux(const FluxParams& P, bool f64, const GridDev* dgrids, int nsm, bool correct, cudaStream_t st);

}  // namespace ovs
