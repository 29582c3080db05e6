// stage_tiles.cu -- the RK3 stage kernels of the launch tuner's other tiles (stage_kernel.cuh) for
// the FP32 forms; a translation unit of its own so that it compiles in parallel with stage.cu.
#include "stage_kernel.cuh"

namespace tgf {

void launch_stage_tile(int tile, int prec, int stage, int mode, int reunit, const Batch& B, const void* w_in,
                       void* w_out, void* acc, void* clov, cudaStream_t st, int grid) {
    if (tile == 1) {
        if (prec == P32) launch_stage_p<P32, 1>(stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
        else launch_stage_p<P32R12, 1>(stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
    } else if (tile == 2) {
        if (prec == P32) launch_stage_p<P32, 2>(stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
        else launch_stage_p<P32R12, 2>(stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
    } else if (tile == 3) {
        if (prec == P32) launch_stage_p<P32, 3>(stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
        else launch_stage_p<P32R12, 3>(stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
    } else {
        if (prec == P32) launch_stage_p<P32, 4>(stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
        else launch_stage_p<P32R12, 4>(stage, mode, reunit, B, w_in, w_out, acc, clov, st, grid);
    }
}

TGF_CHECK_WORD(stage_tiles)

}  // namespace tgf
