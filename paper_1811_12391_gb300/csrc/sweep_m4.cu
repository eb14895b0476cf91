// Instantiations of the octant wavefront sweep for 4 flux moment(s) per cell.
#include "sweep_impl.cuh"

namespace doctors {
cudaError_t launch_sweep_m4_entry(const SweepArgs& a, int mode, cudaStream_t s) {
    switch (mode) {
        case 0: return launch_sweep_m<4, 0>(a, s);
        case 1: return launch_sweep_m<4, 1>(a, s);
        case 2: return launch_sweep_m<4, 2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t upload_tables_m4(const float* R, const float* w) { return upload_direction_tables(R, w); }
}  // namespace doctors
