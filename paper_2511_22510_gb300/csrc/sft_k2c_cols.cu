// sft_k2c_cols.cu -- two-pass 2-D step for complex fields (complex
// Ginzburg-Landau, kernels in sft_k2c.cuh): the column-pass instantiations
// and their size dispatch.
#include "sft_k2c.cuh"

namespace sft {

cudaError_t launch_k2c_cols(const StepArgs& a, int mode, cudaStream_t s) {
    if (a.pshift && mode == MODE_STEP) mode = MODE_STEP_PS;
    if (a.pshift && !a.tw_ps) return cudaErrorInvalidValue;
    switch (a.ny) {
        case 16: return ccols_for<16>(a, mode, s);
        case 32: return ccols_for<32>(a, mode, s);
        case 64: return ccols_for<64>(a, mode, s);
        case 128: return ccols_for<128>(a, mode, s);
        case 256: return ccols_for<256>(a, mode, s);
        case 512: return ccols_for<512>(a, mode, s);
        case 1024: return ccols_for<1024>(a, mode, s);
        case 2048: return ccols_for<2048>(a, mode, s);
        case 4096: return ccols_for<4096>(a, mode, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
