// sft_k2d_cols_large.cu -- column pass of the two-pass 2-D step (kernel in
// sft_k2d_cols.cuh): the instantiations for columns of 512, 1024, 2048 and
// 4096 points (the dispatch of every size is in sft_k2d_cols.cu).
#include "sft_k2d_cols.cuh"

namespace sft {

cudaError_t launch_k2_cols_large(const StepArgs& a, int mode, int nl, cudaStream_t s, int shape) {
    switch (a.ny) {
        case 512: return cols_for<512>(a, mode, nl, s, shape);
        case 1024: return cols_for<1024>(a, mode, nl, s, shape);
        case 2048: return cols_for<2048>(a, mode, nl, s, shape);
        case 4096: return cols_for<4096>(a, mode, nl, s, shape);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
