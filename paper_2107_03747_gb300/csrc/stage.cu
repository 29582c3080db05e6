// stage.cu -- the RK3 stage kernels of the default tile (stage_kernel.cuh) and the launcher that
// dispatches every tile.
#include "stage_kernel.cuh"

namespace tgf {

void launch_stage(int prec, int stage, int mode, int reunit, const Batch& B, const void* w_in, void* w_out,
                  void* acc, void* clov, cudaStream_t st, int grid, int tile) {
    if (tile != 0 && prec != P64 && mode != 2)
        return launch_stage_tile(tile, prec, stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
    if (prec == P64) launch_stage_p<P64, 0>(stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
    else if (prec == P32) launch_stage_p<P32, 0>(stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
    else launch_stage_p<P32R12, 0>(stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
}

TGF_CHECK_WORD(stage)

}  // namespace tgf
