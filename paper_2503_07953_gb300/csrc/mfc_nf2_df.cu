// Directional sweeps for 2 fluid(s) in MODE_DF (double-float WENO5).
#include "mfc_launch_impl.cuh"

namespace mfc {
cudaError_t sweep_df_nf2(const Consts& C, int dir, int mode, SweepArgs A, cudaStream_t s) {
    return sweep_df<2>(C, dir, mode, A, s);
}
}  // namespace mfc
