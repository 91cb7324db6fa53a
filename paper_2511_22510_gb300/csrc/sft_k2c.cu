// sft_k2c.cu -- two-pass 2-D step for complex fields (complex Ginzburg-Landau,
// kernels in sft_k2c.cuh): the row-pass instantiations and their size
// dispatch (the column pass is instantiated in sft_k2c_cols.cu, a
// translation unit of its own, so that the library's units compile in
// parallel in about the same time).
#include "sft_k2c.cuh"

namespace sft {

bool k2c_supported(int nx, int ny) {
    auto ok = [](int n) { return n >= 16 && n <= 4096 && (n & (n - 1)) == 0; };
    return ok(nx) && ok(ny);
}

cudaError_t launch_k2c_rows(const StepArgs& a, int mode, cudaStream_t s) {
    if (mode == MODE_STEP_PS && !a.tw_ps) return cudaErrorInvalidValue;
    switch (a.nx) {
        case 16: return crows_for<16>(a, mode, s);
        case 32: return crows_for<32>(a, mode, s);
        case 64: return crows_for<64>(a, mode, s);
        case 128: return crows_for<128>(a, mode, s);
        case 256: return crows_for<256>(a, mode, s);
        case 512: return crows_for<512>(a, mode, s);
        case 1024: return crows_for<1024>(a, mode, s);
        case 2048: return crows_for<2048>(a, mode, s);
        case 4096: return crows_for<4096>(a, mode, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
