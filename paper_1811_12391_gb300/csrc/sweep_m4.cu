// Instantiations of the octant wavefront sweep for 4 flux moment(s) per cell:
// the tile-stage kernel (k_sweep), the chained kernel (k_sweep_chain) and
// the dataflow kernel (k_sweep_flow).
#include "sweep_flow.cuh"

namespace doctors {
cudaError_t launch_sweep_m4_entry(const SweepArgs& a, int mode, cudaStream_t s) {
    if (a.chain_slots > 0) {
        switch (mode) {
            case 0: return launch_sweep_chain_m<4, 0>(a, s);
            case 1: return launch_sweep_chain_m<4, 1>(a, s);
            case 2: return launch_sweep_chain_m<4, 2>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (mode) {
        case 0: return launch_sweep_m<4, 0>(a, s);
        case 1: return launch_sweep_m<4, 1>(a, s);
        case 2: return launch_sweep_m<4, 2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_sweep_flow_m4_entry(const SweepArgs& a, int mode, cudaStream_t s) {
    switch (mode) {
        case 0: return launch_sweep_flow_m<4, 0>(a, s);
        case 1: return launch_sweep_flow_m<4, 1>(a, s);
        case 2: return launch_sweep_flow_m<4, 2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}
int sweep_flow_blocks_m4(int ab, int threads, size_t smem, bool split, bool dd, bool hw) {
    return sweep_flow_blocks_per_sm<4>(ab, threads, smem, split, dd, hw);
}
cudaError_t launch_split_sweep_m4_entry(const SweepArgs& a, cudaStream_t s, int* count) {
    return launch_split_sweep_m<4>(a, s, count);
}
int sweep_chain_blocks_m4(int ab, bool ct, int threads, size_t smem) { return sweep_chain_blocks_per_sm<4>(ab, ct, threads, smem); }
cudaError_t upload_tables_m4(const float* R, const float* w) {
    cudaError_t e = upload_direction_tables(R, w);
    return e == cudaSuccess ? upload_chain_tables(R, w) : e;
}
}  // namespace doctors
