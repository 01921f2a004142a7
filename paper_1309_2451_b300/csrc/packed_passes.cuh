// packed_passes.cuh -- launchers of the steady complex64 passes in packed
// FP32-pair arithmetic (packed_passes.cu).  Each returns false, launching
// nothing, when the arguments or the geometry are not covered; the caller
// then takes the scalar passes of fast_passes.cu / kernels.cu.
#pragma once

#include "kernels.cuh"

namespace ctap {

// Z pass: nz = 1024, four row classes of four columns per tile (256 x 256
// planes), real time, in place, kinetic (kx, ky) table present
bool packed_z_supported(const Geom &g);
bool launch_z_packed(const ZArgs<float> &a, cudaStream_t st);
// XY pass: nx = 256, 64-row tiles, the steady real-time step with the
// product potential and merged half-kicks, in place
bool packed_xy_supported(const Geom &g);
bool launch_xy_packed(const XYArgs<float> &a, cudaStream_t st);

}  // namespace ctap
