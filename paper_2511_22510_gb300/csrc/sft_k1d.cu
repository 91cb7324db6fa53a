// sft_k1d.cu -- whole-step 1-D kernels (in sft_k1d.cuh): the size dispatch
// and the instantiations for real power-of-two lines.
#include "sft_k1d.cuh"

namespace sft {

// 1-D step variants (MODE_STEP_PS, MODE_STEP_RSN) on power-of-two real lines of up to 16384 points
// (sft_k1d_var.cu)
cudaError_t launch_k1_line_var(const StepArgs& a, int mode, int nl, cudaStream_t s);
// complex lines (sft_k1d_cplx.cu) and the persistent batch kernel (sft_k1d_batch.cu) are translation units of
// their own, so that the library's units compile in parallel in about the same time
cudaError_t launch_k1_line_cplx(const StepArgs& a, int mode, cudaStream_t s);

bool k1_supported(int nx, int complex_field) {
    if (!complex_field && k2_mixed_size(nx)) return true;  // p x 2^k lines (sft_k1d_mixed.cu)
    if ((nx & (nx - 1)) != 0) return false;
    return complex_field ? (nx >= 16 && nx <= 16384) : (nx >= 32 && nx <= 65536);
}

cudaError_t launch_k1_line(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    // complex lines read the N-point table tw_a; real lines the N/2-point table tw_a and the N-point table tw_b
    if (!a.tw_a || (nl != NL_CGL && !a.tw_b)) return cudaErrorInvalidValue;
    if (mode == MODE_STEP_PS || mode == MODE_STEP_RSN) return launch_k1_line_var(a, mode, nl, s);
    if (nl != NL_CGL && k1_use_cluster(a.nx, a.R, mode)) return launch_k1_cluster(a, mode, nl, s);
    if (nl == NL_CGL) return launch_k1_line_cplx(a, mode, s);
    switch (a.nx / 2) {
        case 16: return k1r_for<16>(a, mode, nl, s);
        case 32: return k1r_for<32>(a, mode, nl, s);
        case 64: return k1r_for<64>(a, mode, nl, s);
        case 128: return k1r_for<128>(a, mode, nl, s);
        case 256: return k1r_for<256>(a, mode, nl, s);
        case 512: return k1r_for<512>(a, mode, nl, s);
        case 1024: return k1r_for<1024>(a, mode, nl, s);
        case 2048: return k1r_for<2048>(a, mode, nl, s);
        case 4096: return k1r_for<4096>(a, mode, nl, s);
        case 8192: return k1r_for<8192>(a, mode, nl, s);
        case 16384: return k1r_for<16384>(a, mode, nl, s);
        default: return k2_mixed_size(a.nx) ? launch_k1_line_mixed(a, mode, nl, s) : cudaErrorInvalidValue;
    }
}

}  // namespace sft
