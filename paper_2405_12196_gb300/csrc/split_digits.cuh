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

// The float 2^23 + b for 0 <= b < 2^23: b in the low mantissa bits of 2^23.
__device__ __forceinline__ float biased_int(uint32_t b) { return __uint_as_float(0x4B000000u | b); }

// Byte k of x as the float 2^23 + byte (one byte permute).
template <int K>
__device__ __forceinline__ float biased_byte(uint32_t x) {
  return __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7540u | K));
}

// Two floats with at most 8 significant bits as a BF16 pair (low half: f0). Their
// BF16 values are exact: the upper 16 bits of each float.
__device__ __forceinline__ uint32_t pack_exact_bf16(float f0, float f1) {
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632u);
}

// Eight consecutive elements of one row (raw FP64 bits) -> s slices of 8 BF16
// values each, packed as 16 bytes per slice (two elements per 32-bit word, the
// even one in the low half).
__device__ __forceinline__ void slice_digits8(const unsigned long long *bits8, int e, int s,
                                              uint32_t (&packed)[kSlices][4]) {
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    uint32_t lo[2], hi[2];
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
      // below the s kept digits are 128, i.e. digits 0.
      const unsigned long long w = ((unsigned long long)u << (8 * (kSlices - s))) + 0x808080808080ull;
      lo[h] = (uint32_t)w;
      hi[h] = (uint32_t)(w >> 32);
    }
    // slice p holds d_p 2^(-8p) = (byte - 128) 2^(-8p): from the float 2^23 + byte,
    // one exact FMA ((2^23 + byte) 2^(-8p) - (2^23 + 128) 2^(-8p), both terms and
    // the result representable); the leading digit (up to 256 - 128) one exact add
    constexpr float kBias = 8388608.0f + 128.0f;
    packed[0][j >> 1] = pack_exact_bf16(biased_int(hi[0] >> 8) - kBias, biased_int(hi[1] >> 8) - kBias);
    if (s > 1)
      packed[1][j >> 1] = pack_exact_bf16(fmaf(biased_byte<0>(hi[0]), 0x1p-8f, -kBias * 0x1p-8f),
                                          fmaf(biased_byte<0>(hi[1]), 0x1p-8f, -kBias * 0x1p-8f));
    if (s > 2)
      packed[2][j >> 1] = pack_exact_bf16(fmaf(biased_byte<3>(lo[0]), 0x1p-16f, -kBias * 0x1p-16f),
                                          fmaf(biased_byte<3>(lo[1]), 0x1p-16f, -kBias * 0x1p-16f));
    if (s > 3)
      packed[3][j >> 1] = pack_exact_bf16(fmaf(biased_byte<2>(lo[0]), 0x1p-24f, -kBias * 0x1p-24f),
                                          fmaf(biased_byte<2>(lo[1]), 0x1p-24f, -kBias * 0x1p-24f));
    if (s > 4)
      packed[4][j >> 1] = pack_exact_bf16(fmaf(biased_byte<1>(lo[0]), 0x1p-32f, -kBias * 0x1p-32f),
                                          fmaf(biased_byte<1>(lo[1]), 0x1p-32f, -kBias * 0x1p-32f));
    if (s > 5)
      packed[5][j >> 1] = pack_exact_bf16(fmaf(biased_byte<0>(lo[0]), 0x1p-40f, -kBias * 0x1p-40f),
                                          fmaf(biased_byte<0>(lo[1]), 0x1p-40f, -kBias * 0x1p-40f));
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
