// sft_k2d_cols.cu -- column pass of the two-pass 2-D step (kernel in
// sft_k2d_cols.cuh): the power-of-two instantiations and the size dispatch.
#include "sft_k2d_cols.cuh"

namespace sft {

bool k2_mixed_size(int n) {
    for (int p : {3, 5, 7})
        if (n % p == 0 && ((n / p) & (n / p - 1)) == 0) return n >= 16 * p && n <= 768;
    return false;
}

bool k2_supported(int nx, int ny, int complex_field) {
    if (complex_field) return false;
    auto ok = [](int n) { return (n >= 16 && n <= 4096 && (n & (n - 1)) == 0) || k2_mixed_size(n); };
    return ok(nx) && ok(ny);
}

// shapes 0-2: the radix schedules and block shapes of k2_cols_real; 3 (columns of 1024 points): one warp
// per column, sft_k2d_colwarp.cu (cubic term, see k2_colwarp_supported)
int k2_col_shapes(int ny) { return (ny & (ny - 1)) == 0 && ny >= 512 ? (ny == 1024 ? 4 : 3) : 1; }

// columns of 512 to 4096 points: sft_k2d_cols_large.cu (a translation unit of its own, so that the
// library's units compile in parallel in about the same time)
cudaError_t launch_k2_cols_large(const StepArgs& a, int mode, int nl, cudaStream_t s, int shape);

cudaError_t launch_k2_cols(const StepArgs& a, int mode, int nl, cudaStream_t s, int shape) {
    if (shape == 3 && mode == MODE_STEP && !a.rec_phi && !a.noise_in && !a.pshift) return launch_k2_cols_warp(a, nl, s);
    switch (a.ny) {
        case 16: return cols_for<16>(a, mode, nl, s, shape);
        case 32: return cols_for<32>(a, mode, nl, s, shape);
        case 64: return cols_for<64>(a, mode, nl, s, shape);
        case 128: return cols_for<128>(a, mode, nl, s, shape);
        case 256: return cols_for<256>(a, mode, nl, s, shape);
        case 512:
        case 1024:
        case 2048:
        case 4096: return launch_k2_cols_large(a, mode, nl, s, shape);
        default: return k2_mixed_size(a.ny) ? launch_k2_cols_mixed(a, mode, nl, s) : cudaErrorInvalidValue;
    }
}

}  // namespace sft
