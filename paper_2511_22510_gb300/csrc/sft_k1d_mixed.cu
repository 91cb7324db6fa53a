// sft_k1d_mixed.cu -- whole-step 1-D kernels on real lines of p x 2^k points,
// p in {3, 5, 7} (the radix-p plans of FftPlan): transforms and the step.
#include "sft_k1d.cuh"

namespace sft {

template <int M>
static cudaError_t k1r_for_mixed(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    if (mode == MODE_FWD) return run_k1_real<M, NL_CUBIC, MODE_FWD>(a, s);
    if (mode == MODE_INV) return run_k1_real<M, NL_CUBIC, MODE_INV>(a, s);
    if (mode == MODE_STEP && nl == NL_CUBIC) return run_k1_real<M, NL_CUBIC, MODE_STEP>(a, s);
    if (mode == MODE_STEP && nl == NL_GRAD2) return run_k1_real<M, NL_GRAD2, MODE_STEP>(a, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_k1_line_mixed(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    switch (a.nx / 2) {
        case 24: return k1r_for_mixed<24>(a, mode, nl, s);
        case 48: return k1r_for_mixed<48>(a, mode, nl, s);
        case 96: return k1r_for_mixed<96>(a, mode, nl, s);
        case 192: return k1r_for_mixed<192>(a, mode, nl, s);
        case 384: return k1r_for_mixed<384>(a, mode, nl, s);
        case 40: return k1r_for_mixed<40>(a, mode, nl, s);
        case 80: return k1r_for_mixed<80>(a, mode, nl, s);
        case 160: return k1r_for_mixed<160>(a, mode, nl, s);
        case 320: return k1r_for_mixed<320>(a, mode, nl, s);
        case 56: return k1r_for_mixed<56>(a, mode, nl, s);
        case 112: return k1r_for_mixed<112>(a, mode, nl, s);
        case 224: return k1r_for_mixed<224>(a, mode, nl, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
