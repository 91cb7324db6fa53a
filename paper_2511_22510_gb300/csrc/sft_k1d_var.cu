// sft_k1d_var.cu -- the 1-D step variants (phase-shift dealiasing, real-space
// noise; the alternatives of Sec. IV steps 1 and 2) on power-of-two real lines
// of up to 16384 points: the instantiations of k1_real's MODE_STEP_PS and
// MODE_STEP_RSN (sft_k1d.cuh), in a translation unit of their own so that the
// build compiles them in parallel with the plain line kernels.
#include "sft_k1d.cuh"

namespace sft {

template <int M>
static cudaError_t k1r_var(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    if (mode == MODE_STEP_PS && nl == NL_CUBIC) return run_k1_real<M, NL_CUBIC, MODE_STEP_PS>(a, s);
    if (mode == MODE_STEP_PS && nl == NL_GRAD2) return run_k1_real<M, NL_GRAD2, MODE_STEP_PS>(a, s);
    if (mode == MODE_STEP_RSN && nl == NL_CUBIC) return run_k1_real<M, NL_CUBIC, MODE_STEP_RSN>(a, s);
    if (mode == MODE_STEP_RSN && nl == NL_GRAD2) return run_k1_real<M, NL_GRAD2, MODE_STEP_RSN>(a, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_k1_line_var(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    if (mode == MODE_STEP_PS && !a.tw_ps) return cudaErrorInvalidValue;
    switch (a.nx / 2) {
        case 16: return k1r_var<16>(a, mode, nl, s);
        case 32: return k1r_var<32>(a, mode, nl, s);
        case 64: return k1r_var<64>(a, mode, nl, s);
        case 128: return k1r_var<128>(a, mode, nl, s);
        case 256: return k1r_var<256>(a, mode, nl, s);
        case 512: return k1r_var<512>(a, mode, nl, s);
        case 1024: return k1r_var<1024>(a, mode, nl, s);
        case 2048: return k1r_var<2048>(a, mode, nl, s);
        case 4096: return k1r_var<4096>(a, mode, nl, s);
        case 8192: return k1r_var<8192>(a, mode, nl, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
