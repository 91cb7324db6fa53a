// sft_k1d_cplx.cu -- whole-step 1-D kernels (in sft_k1d.cuh) on complex
// lines (CGL) of 16 to 16384 points: the instantiations and the size dispatch.
#include "sft_k1d.cuh"

namespace sft {

cudaError_t launch_k1_line_cplx(const StepArgs& a, int mode, cudaStream_t s) {
    switch (a.nx) {
        case 16: return k1c_for<16>(a, mode, s);
        case 32: return k1c_for<32>(a, mode, s);
        case 64: return k1c_for<64>(a, mode, s);
        case 128: return k1c_for<128>(a, mode, s);
        case 256: return k1c_for<256>(a, mode, s);
        case 512: return k1c_for<512>(a, mode, s);
        case 1024: return k1c_for<1024>(a, mode, s);
        case 2048: return k1c_for<2048>(a, mode, s);
        case 4096: return k1c_for<4096>(a, mode, s);
        case 8192: return k1c_for<8192>(a, mode, s);
        case 16384: return k1c_for<16384>(a, mode, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
