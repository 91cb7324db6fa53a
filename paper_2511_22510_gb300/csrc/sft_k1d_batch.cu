// sft_k1d_batch.cu -- the persistent batch kernel of the whole-step 1-D
// kernels (in sft_k1d.cuh): every 1-D member of a batch of up to 8192-point
// half-spectra in one launch.
#include "sft_k1d.cuh"

namespace sft {

// ------------------------------------------------------------------ batches
// One persistent launch advances every replica of every 1-D member of a batch
// by one step: each block takes work items (member, first replica) from a
// device queue (largest lattices first) and runs the size's line_step with as
// many teams as fit its 512 threads.  Lattices up to 16384 points (line
// teams of at most 512 threads).
constexpr int kBatchThreads = 512;
template <int M>
struct BatchLines {
    static constexpr int T = FftPlan<M>::T;
    static constexpr int LINES = kBatchThreads / T;
    static constexpr int XB = FftPlan<M>::BUF;
};

template <int M, int NL>
__device__ __forceinline__ void batch_lines(const StepArgs& a, int r0, float2* sm) {
    using B = BatchLines<M>;
    const int team = threadIdx.x / B::T, t = threadIdx.x % B::T;
    if (team >= B::LINES) return;  // whole teams idle
    const int r = r0 + team;
    const bool valid = r < a.R;
    line_step<M, NL>(a, valid ? r : a.R - 1, valid, t, sm + team * B::XB);
}

template <int NL>
__global__ void __launch_bounds__(kBatchThreads, 1)
    k1_batch(const BatchMember* __restrict__ members, const BatchItem* __restrict__ items, int nitems, int* head,
             int k_in_chunk) {
    extern __shared__ float2 sm[];
    __shared__ int cur;
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(head, 1);
        __syncthreads();
        const int it = cur;
        __syncthreads();
        if (it >= nitems) break;
        const BatchItem w = items[it];
        StepArgs a = members[w.member].a;
        a.k_in_chunk = k_in_chunk;
        switch (members[w.member].M) {
            case 16: batch_lines<16, NL>(a, w.r0, sm); break;
            case 32: batch_lines<32, NL>(a, w.r0, sm); break;
            case 64: batch_lines<64, NL>(a, w.r0, sm); break;
            case 128: batch_lines<128, NL>(a, w.r0, sm); break;
            case 256: batch_lines<256, NL>(a, w.r0, sm); break;
            case 512: batch_lines<512, NL>(a, w.r0, sm); break;
            case 1024: batch_lines<1024, NL>(a, w.r0, sm); break;
            case 2048: batch_lines<2048, NL>(a, w.r0, sm); break;
            case 4096: batch_lines<4096, NL>(a, w.r0, sm); break;
            case 8192: batch_lines<8192, NL>(a, w.r0, sm); break;
            default: break;
        }
        __syncthreads();
    }
}

int batch_lines_per_item(int M) {
    switch (M) {
        case 16: return BatchLines<16>::LINES;
        case 32: return BatchLines<32>::LINES;
        case 64: return BatchLines<64>::LINES;
        case 128: return BatchLines<128>::LINES;
        case 256: return BatchLines<256>::LINES;
        case 512: return BatchLines<512>::LINES;
        case 1024: return BatchLines<1024>::LINES;
        case 2048: return BatchLines<2048>::LINES;
        case 4096: return BatchLines<4096>::LINES;
        case 8192: return BatchLines<8192>::LINES;
        default: return 0;
    }
}

size_t batch_smem_bytes() {
    size_t b = 0;
    auto upd = [&](size_t v) { b = v > b ? v : b; };
    upd(sizeof(float2) * BatchLines<16>::LINES * BatchLines<16>::XB);
    upd(sizeof(float2) * BatchLines<32>::LINES * BatchLines<32>::XB);
    upd(sizeof(float2) * BatchLines<64>::LINES * BatchLines<64>::XB);
    upd(sizeof(float2) * BatchLines<128>::LINES * BatchLines<128>::XB);
    upd(sizeof(float2) * BatchLines<256>::LINES * BatchLines<256>::XB);
    upd(sizeof(float2) * BatchLines<512>::LINES * BatchLines<512>::XB);
    upd(sizeof(float2) * BatchLines<1024>::LINES * BatchLines<1024>::XB);
    upd(sizeof(float2) * BatchLines<2048>::LINES * BatchLines<2048>::XB);
    upd(sizeof(float2) * BatchLines<4096>::LINES * BatchLines<4096>::XB);
    upd(sizeof(float2) * BatchLines<8192>::LINES * BatchLines<8192>::XB);
    return b;
}

cudaError_t launch_k1_batch(const BatchMember* members, const BatchItem* items, int nitems, int* head, int nl,
                            int k_in_chunk, int blocks, cudaStream_t s) {
    static bool attr[2] = {false, false};
    const size_t sm = batch_smem_bytes();
    const int which = nl == NL_GRAD2 ? 1 : 0;
    if (!attr[which]) {
        cudaError_t e = which ? cudaFuncSetAttribute(k1_batch<NL_GRAD2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)sm)
                              : cudaFuncSetAttribute(k1_batch<NL_CUBIC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)sm);
        if (e != cudaSuccess) return e;
        attr[which] = true;
    }
    if (which)
        k1_batch<NL_GRAD2><<<blocks, kBatchThreads, sm, s>>>(members, items, nitems, head, k_in_chunk);
    else
        k1_batch<NL_CUBIC><<<blocks, kBatchThreads, sm, s>>>(members, items, nitems, head, k_in_chunk);
    return cudaGetLastError();
}

}  // namespace sft
