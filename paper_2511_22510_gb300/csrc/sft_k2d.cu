// sft_k2d.cu -- row pass of the two-pass 2-D step (kernel in sft_k2d.cuh):
// the power-of-two instantiations and the size dispatch.
#include "sft_k2d.cuh"

namespace sft {

// (the forward transform of the real-space noise is instantiated here, for power-of-two rows)
// shapes 0-2: the block shapes of k2_rows_real; 3 (rows of 1024 points): the two-rows-per-warp kernel of
// sft_k2d_pair.cu (cubic term, see k2_pair_supported)
int k2_row_shapes(int nx) { return (nx & (nx - 1)) == 0 ? (nx == 1024 ? 4 : 3) : 1; }

// rows of 1024 to 4096 points: sft_k2d_large.cu (a translation unit of its own, so that the library's units
// compile in parallel in about the same time)
cudaError_t launch_k2_rows_large(const StepArgs& a, int mode, int nl, cudaStream_t s, int shape);

cudaError_t launch_k2_rows(const StepArgs& a, int mode, int nl, cudaStream_t s, int shape) {
    if (shape == 3) return mode == MODE_STEP ? launch_k2_rows_pair(a, nl, s) : cudaErrorInvalidValue;
    switch (a.nx / 2) {
        case 8: return rows_for<8>(a, mode, nl, s, shape);
        case 16: return rows_for<16>(a, mode, nl, s, shape);
        case 32: return rows_for<32>(a, mode, nl, s, shape);
        case 64: return rows_for<64>(a, mode, nl, s, shape);
        case 128: return rows_for<128>(a, mode, nl, s, shape);
        case 256: return rows_for<256>(a, mode, nl, s, shape);
        case 512:
        case 1024:
        case 2048: return launch_k2_rows_large(a, mode, nl, s, shape);
        default: return k2_mixed_size(a.nx) ? launch_k2_rows_mixed(a, mode, nl, s) : cudaErrorInvalidValue;
    }
}

}  // namespace sft
