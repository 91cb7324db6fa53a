// sft_k2d_mixed.cu -- row pass on rows of p x 2^k points, p in {3, 5, 7}
// (the radix-p plans of FftPlan): transforms and the step.
#include "sft_k2d.cuh"

namespace sft {

// Rows of M = p x 2^k points, p in {3, 5, 7} (lattices of 16p .. 768 points): transforms and the
// step (default schedule).
template <int M>
static cudaError_t rows_for_mixed(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    if (mode == MODE_FWD) return run_rows<M, NL_CUBIC, MODE_FWD>(a, s);
    if (mode == MODE_INV) return run_rows<M, NL_CUBIC, MODE_INV>(a, s);
    if (mode == MODE_STEP && nl == NL_CUBIC) return run_rows<M, NL_CUBIC, MODE_STEP>(a, s);
    if (mode == MODE_STEP && nl == NL_GRAD2) return run_rows<M, NL_GRAD2, MODE_STEP>(a, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_k2_rows_mixed(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    switch (a.nx / 2) {
        case 24: return rows_for_mixed<24>(a, mode, nl, s);
        case 48: return rows_for_mixed<48>(a, mode, nl, s);
        case 96: return rows_for_mixed<96>(a, mode, nl, s);
        case 192: return rows_for_mixed<192>(a, mode, nl, s);
        case 384: return rows_for_mixed<384>(a, mode, nl, s);
        case 40: return rows_for_mixed<40>(a, mode, nl, s);
        case 80: return rows_for_mixed<80>(a, mode, nl, s);
        case 160: return rows_for_mixed<160>(a, mode, nl, s);
        case 320: return rows_for_mixed<320>(a, mode, nl, s);
        case 56: return rows_for_mixed<56>(a, mode, nl, s);
        case 112: return rows_for_mixed<112>(a, mode, nl, s);
        case 224: return rows_for_mixed<224>(a, mode, nl, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
