// sft_warpfft.cuh -- 1024-point complex FFT held by one warp in registers
// (32 values per lane), and the TMA (cp.async.bulk.tensor) wrappers used by
// the kernels built on it.
//
// Index split n = t + 32 e (lane t, slot e), k = k1 + 32 k2:
//   X[k1 + 32 k2] = sum_t W_32^{t k2} W_1024^{t k1} [ sum_e x[t + 32 e] W_32^{e k1} ]
// Pass A: a 32-point DFT over the slots of each lane; twiddle W_1024^{t k1};
// one 32 x 32 transpose through a swizzled 8 KB shared-memory buffer; pass B:
// a 32-point DFT over the lanes.  Input and output use the same layout (lane
// t, slot e holds index t + 32 e), so transforms can be chained in registers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sft_async.cuh"
#include "sft_device.cuh"

namespace sft {

// Complex sum and difference with the paired single-precision instructions of
// sm_100 and later (one instruction for both components).
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// 32-point DFT in registers (radix-2 decimation in frequency, then the
// bit-reversal permutation resolved at compile time).  ZIN marks inputs known
// to be zero: the first stage skips the additions they would take part in.
template <bool INV, uint32_t ZIN>
__device__ __forceinline__ void dft32(float2 (&x)[32]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const bool za = (ZIN >> i) & 1u, zb = (ZIN >> (i + 16)) & 1u;
        const float2 a = x[i], b = x[i + 16];
        if (za && zb) {
            x[i] = czero();
            x[i + 16] = czero();
        } else if (za) {
            x[i] = b;
            x[i + 16] = twiddle_const<INV>(make_float2(-b.x, -b.y), i, 32);
        } else if (zb) {
            x[i] = a;
            x[i + 16] = twiddle_const<INV>(a, i, 32);
        } else {
            x[i] = padd(a, b);
            x[i + 16] = twiddle_const<INV>(psub(a, b), i, 32);
        }
    }
#pragma unroll
    for (int span = 8; span >= 1; span >>= 1) {
#pragma unroll
        for (int blk = 0; blk < 32; blk += 2 * span) {
#pragma unroll
            for (int i = 0; i < span; ++i) {
                const float2 a = x[blk + i], b = x[blk + i + span];
                x[blk + i] = padd(a, b);
                x[blk + i + span] = twiddle_const<INV>(psub(a, b), i * (16 / span), 32);
            }
        }
    }
    float2 y[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) y[k] = x[bitrev<32>(k)];
#pragma unroll
    for (int k = 0; k < 32; ++k) x[k] = y[k];
}

// Twiddle W_1024^{+-t k1} of pass A, then the transpose: lane t hands slot k1
// to lane k1, which receives slot t.  xb: the warp's 1024-element buffer;
// element (t, k1) sits at t 32 + (k1 ^ (2t mod 32)), so the 16-byte stores of
// a quarter warp and the 8-byte loads of a half warp are free of bank
// conflicts.  tw32[k1 32 + t] = W_1024^{t k1} (forward sign).  Ten exact
// table entries per lane, S_j = W^{t j} (j < 8) and B_g = W^{8 g t}, give every
// twiddle of slot k1 = 8 g + j as a multiplication by S_j and then by B_g:
// fewer live registers than one load per slot or a table of products.
template <bool INV>
__device__ __forceinline__ void warp_twiddle_transpose(float2 (&v)[32], float2* xb, int lane,
                                                       const float2* __restrict__ tw32) {
    // the table address passes through an empty asm that depends on the DFT outputs, so that the
    // loads are issued after pass A and not hoisted (or shared between transforms) ahead of it
    const float2* tw = tw32;
    asm volatile("" : "+l"(tw) : "f"(v[0].x), "f"(v[31].y));
    float2 S[8], B[4];
#pragma unroll
    for (int j = 1; j < 8; ++j) {
        S[j] = __ldg(&tw[j * 32 + lane]);
        if (INV) S[j].y = -S[j].y;
    }
#pragma unroll
    for (int g = 1; g < 4; ++g) {
        B[g] = __ldg(&tw[8 * g * 32 + lane]);
        if (INV) B[g].y = -B[g].y;
    }
#pragma unroll
    for (int k1 = 1; k1 < 32; ++k1) {
        const int g = k1 >> 3, j = k1 & 7;
        if (j) v[k1] = cmul(v[k1], S[j]);
        if (g) v[k1] = cmul(v[k1], B[g]);
    }
    __syncwarp();
    const int s = (2 * lane) & 31;
    float2* row = xb + lane * 32;
#pragma unroll
    for (int k1 = 0; k1 < 32; k1 += 2)
        *reinterpret_cast<float4*>(row + (k1 ^ s)) = make_float4(v[k1].x, v[k1].y, v[k1 + 1].x, v[k1 + 1].y);
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 32; ++t) v[t] = xb[t * 32 + (lane ^ ((2 * t) & 31))];
    __syncwarp();
}

// Unnormalised 1024-point FFT (forward e^{-2 pi i}, inverse e^{+2 pi i}) of the
// line held by the warp: v[e] of lane t is x[t + 32 e] on entry and X[t + 32 e]
// on exit.  ZIN: slots e that are zero in every lane on entry.
template <bool INV, uint32_t ZIN = 0u>
__device__ __forceinline__ void fft1024_warp(float2 (&v)[32], float2* xb, int lane, const float2* __restrict__ tw32) {
    dft32<INV, ZIN>(v);
    warp_twiddle_transpose<INV>(v, xb, lane, tw32);
    dft32<INV, 0u>(v);
}

// ------------------------------------------------------------------ TMA
// 3-D tiled copies through a tensor map passed as a __grid_constant__ kernel
// parameter.  The innermost coordinate x, times the element size, must be a
// multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(void* dst_smem, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst_smem)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, const void* src_smem) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(smem_addr(src_smem))
                 : "memory");
}

__device__ __forceinline__ void tma_store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until every committed store has finished reading shared memory
__device__ __forceinline__ void tma_store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

}  // namespace sft
