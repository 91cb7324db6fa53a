// sft_k2d_cols_mixed.cu -- column pass on columns of p x 2^k points, p in
// {3, 5, 7} (the radix-p plans of FftPlan): transforms, the step and P.
#include "sft_k2d_cols.cuh"

namespace sft {

// Columns of NY = p x 2^k points, p in {3, 5, 7} (16p .. 768): transforms, the step and P (default schedule).
template <int NY>
static cudaError_t cols_for_mixed(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    if (mode == MODE_FWD) return run_cols<NY, NL_CUBIC, MODE_FWD>(a, s);
    if (mode == MODE_INV) return run_cols<NY, NL_CUBIC, MODE_INV>(a, s);
    if (mode == MODE_STEP && nl == NL_CUBIC) return run_cols<NY, NL_CUBIC, MODE_STEP>(a, s);
    if (mode == MODE_STEP && nl == NL_GRAD2) return run_cols<NY, NL_GRAD2, MODE_STEP>(a, s);
    if (mode == MODE_PRIME && nl == NL_CUBIC) return run_cols<NY, NL_CUBIC, MODE_PRIME>(a, s);
    if (mode == MODE_PRIME && nl == NL_GRAD2) return run_cols<NY, NL_GRAD2, MODE_PRIME>(a, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_k2_cols_mixed(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    switch (a.ny) {
        case 48: return cols_for_mixed<48>(a, mode, nl, s);
        case 96: return cols_for_mixed<96>(a, mode, nl, s);
        case 192: return cols_for_mixed<192>(a, mode, nl, s);
        case 384: return cols_for_mixed<384>(a, mode, nl, s);
        case 768: return cols_for_mixed<768>(a, mode, nl, s);
        case 80: return cols_for_mixed<80>(a, mode, nl, s);
        case 160: return cols_for_mixed<160>(a, mode, nl, s);
        case 320: return cols_for_mixed<320>(a, mode, nl, s);
        case 640: return cols_for_mixed<640>(a, mode, nl, s);
        case 112: return cols_for_mixed<112>(a, mode, nl, s);
        case 224: return cols_for_mixed<224>(a, mode, nl, s);
        case 448: return cols_for_mixed<448>(a, mode, nl, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
