// Digits of the error-free split (shared by the staged and the fused slice
// kernels). For an element x of a row with scale 2^e (|x| < 2^(e - 1)), the
// integer u = round(x 2^(8s - e)), |u| <= 2^(8s - 1), is written in balanced base
// 256, u = sum_{p < s} d_p 256^(s - 1 - p) with d_p in [-128, 127] (the leading
// one in [-128, 128]); slice p holds d_p 2^(-8p). The digits come from the FP64
// bit pattern with integer operations only.
#pragma once

#include <cuda_bf16.h>

#include "ytn_internal.hpp"

namespace ytn {

static_assert(kSlices == 6, "the digits are taken from fixed byte positions");

// Eight consecutive elements of one row (raw FP64 bits) -> s slices of 8 BF16
// values each, packed as 16 bytes per slice (two elements per 32-bit word, the
// even one in the low half).
__device__ __forceinline__ void slice_digits8(const unsigned long long *bits8, int e, int s,
                                              uint32_t (&packed)[kSlices][4]) {
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    float f[2][kSlices];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const unsigned long long bits = bits8[j + h];
      const int Eb = (int)((bits >> 52) & 0x7FF);
      // |u| = round(|x| 2^-e 2^(8s)) <= 2^(8s-1): the s kept digits, rounded to nearest
      long long u = 0;
      if (Eb != 0) {
        const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int shift = 1075 + e - Eb - 8 * s;   // >= 54 - 8s >= 6
        if (shift < 64) u = (long long)((mant + (1ull << (shift - 1))) >> shift);
        if (bits >> 63) u = -u;
      }
      // balanced base-256 digits: with w = u 256^(6-s) + sum_q 128 256^q (q < 6),
      // digit p (most significant first) is byte 5 - p of w minus 128, the leading
      // one taking the carry above byte 5 as well (it lies in [-128, 128]); bytes
      // below the s kept digits are 128, i.e. digits 0. Each slice value
      // d_p 2^(-8p) = byte 2^(-8p) - 128 2^(-8p) is one exact FMA.
      const unsigned long long w = ((unsigned long long)u << (8 * (kSlices - s))) + 0x808080808080ull;
      const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
      f[h][0] = (float)(hi >> 8) - 128.0f;
      f[h][1] = fmaf((float)(hi & 255u), 0x1p-8f, -0x1p-1f);
      f[h][2] = fmaf((float)(lo >> 24), 0x1p-16f, -0x1p-9f);
      f[h][3] = fmaf((float)((lo >> 16) & 255u), 0x1p-24f, -0x1p-17f);
      f[h][4] = fmaf((float)((lo >> 8) & 255u), 0x1p-32f, -0x1p-25f);
      f[h][5] = fmaf((float)(lo & 255u), 0x1p-40f, -0x1p-33f);
    }
#pragma unroll
    for (int p = 0; p < kSlices; p++) {
      const __nv_bfloat162 pr = __floats2bfloat162_rn(f[0][p], f[1][p]);
      packed[p][j >> 1] = *reinterpret_cast<const uint32_t *>(&pr);
    }
  }
}

// Position of row rr's 16-byte chunk c (8 elements of K) inside a 128 x 32 slice:
// K-major, 64 bytes per row, chunk c stored at c ^ ((rr >> 1) & 3) (the 64-byte
// swizzle the tensor cores read).
__device__ __forceinline__ int slice_pos(int rr, int c) { return rr * 64 + ((c ^ ((rr >> 1) & 3)) << 4); }

__device__ __forceinline__ void store_slices(uint8_t *blk, int pos, int s, const uint32_t (&packed)[kSlices][4]) {
#pragma unroll
  for (int p = 0; p < kSlices; p++)
    if (p < s)   // slices beyond s are never read
      *reinterpret_cast<uint4 *>(blk + p * kSliceBytes + pos) =
          make_uint4(packed[p][0], packed[p][1], packed[p][2], packed[p][3]);
}

__device__ __forceinline__ int biased_exp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

}  // namespace ytn
