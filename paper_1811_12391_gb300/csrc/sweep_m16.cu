// Instantiations of the octant wavefront sweep for 16 flux moment(s) per cell:
// the tile-stage kernel (k_sweep), the chained kernel (k_sweep_chain) and
// the dataflow kernel (k_sweep_flow).
#include "sweep_flow.cuh"

namespace doctors {
cudaError_t launch_sweep_m16_entry(const SweepArgs& a, int mode, cudaStream_t s) {
    if (a.chain_slots > 0) {
        switch (mode) {
            case 0: return launch_sweep_chain_m<16, 0>(a, s);
            case 1: return launch_sweep_chain_m<16, 1>(a, s);
            case 2: return launch_sweep_chain_m<16, 2>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (mode) {
        case 0: return launch_sweep_m<16, 0>(a, s);
        case 1: return launch_sweep_m<16, 1>(a, s);
        case 2: return launch_sweep_m<16, 2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_sweep_flow_m16_entry(const SweepArgs& a, int mode, cudaStream_t s) {
    switch (mode) {
        case 0: return launch_sweep_flow_m<16, 0>(a, s);
        case 1: return launch_sweep_flow_m<16, 1>(a, s);
        case 2: return launch_sweep_flow_m<16, 2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}
int sweep_flow_blocks_m16(int ab, int threads, size_t smem, bool split, bool dd, bool hw) {
    return sweep_flow_blocks_per_sm<16>(ab, threads, smem, split, dd, hw);
}
cudaError_t launch_split_sweep_m16_entry(const SweepArgs& a, cudaStream_t s, int* count) {
    return launch_split_sweep_m<16>(a, s, count);
}
int sweep_chain_blocks_m16(int ab, bool ct, int threads, size_t smem) { return sweep_chain_blocks_per_sm<16>(ab, ct, threads, smem); }
cudaError_t upload_tables_m16(const float* R, const float* w) {
    cudaError_t e = upload_direction_tables(R, w);
    return e == cudaSuccess ? upload_chain_tables(R, w) : e;
}
}  // namespace doctors
