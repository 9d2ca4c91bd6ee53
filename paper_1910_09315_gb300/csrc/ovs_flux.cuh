// Contravariant fluxes at the receivers and the mass-conservation correction (see ovs_flux.cu).
#pragma once
#include <algorithm>

#include "ovs_internal.cuh"

namespace ovs {

constexpr int kMaxFluxSurfaces = 64;
// partial sums of a call: at most this many chunks of consecutive surface faces (the context workspace holds
// their (net, area) pairs)
constexpr int kFluxChunks = 4096;

struct FluxParams {
    int32_t grid;
    int32_t nsurf;
    int64_t nfaces;
    const int64_t* faces;  // face id = 3 * base node + d
    const int8_t* signs;   // +1 / -1 per face (NULL: all +1)
    FieldsDev vel;         // node velocities u, v, w of the grid
    void* flux;            // [nfaces], the fields' type
    double* net;           // [2 nsurf]: net signed flux before the correction, total face area
    double* part;          // [2 kFluxChunks]: (net, area) of each chunk (context workspace)
    int32_t* err;
    int32_t chunk;                              // faces per chunk (a multiple of 256)
    int64_t surf_start[kMaxFluxSurfaces + 1];
    int32_t chunk_start[kMaxFluxSurfaces + 1];  // surface s owns chunks chunk_start[s] .. chunk_start[s+1]-1
};

cudaError_t launch_flux(const FluxParams& P, bool f64, const GridDev* dgrids, int nsm, bool correct, cudaStream_t st);

}  // namespace ovs
