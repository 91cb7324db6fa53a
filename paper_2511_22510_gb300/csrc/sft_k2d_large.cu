// sft_k2d_large.cu -- row pass of the two-pass 2-D step (kernel in
// sft_k2d.cuh): the instantiations for rows of 1024, 2048 and 4096 points
// (half-spectra of 512 to 2048 modes; the dispatch of every size is in
// sft_k2d.cu).
#include "sft_k2d.cuh"

namespace sft {

cudaError_t launch_k2_rows_large(const StepArgs& a, int mode, int nl, cudaStream_t s, int shape) {
    switch (a.nx / 2) {
        case 512: return rows_for<512>(a, mode, nl, s, shape);
        case 1024: return rows_for<1024>(a, mode, nl, s, shape);
        case 2048: return rows_for<2048>(a, mode, nl, s, shape);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
