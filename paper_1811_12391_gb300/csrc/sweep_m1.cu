// Instantiations of the octant wavefront sweep for 1 flux moment(s) per cell.
#include "sweep_impl.cuh"

namespace doctors {
cudaError_t launch_sweep_m1_entry(const SweepArgs& a, cudaStream_t s) { return launch_sweep_m<1>(a, s); }
}  // namespace doctors
