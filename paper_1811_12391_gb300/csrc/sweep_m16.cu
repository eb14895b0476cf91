// Instantiations of the octant wavefront sweep for 16 flux moment(s) per cell.
#include "sweep_impl.cuh"

namespace doctors {
cudaError_t launch_sweep_m16_entry(const SweepArgs& a, cudaStream_t s) { return launch_sweep_m<16>(a, s); }
}  // namespace doctors
