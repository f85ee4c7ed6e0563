// Two x-adjacent points per thread: storage access and the BCC pull gather
// for a pair (x0, x0 + 1), x0 even, of the same (y, z, sublattice) (Sec. 5).
//
// A pair of stored populations is one aligned 8-byte (FP32) or 4-byte
// (16-bit) word. A pull whose x shift is even reads one such word; an odd
// shift straddles two words and takes the upper element of the lower word and
// the lower element of the upper word. Every source of a pair therefore lies
// in the three pair columns x0/2 - 1, x0/2, x0/2 + 1 (periodic in x; nx even).
#pragma once

#include "rpk_device.cuh"

namespace rpk {

// pair word <-> two FP32 values
template <typename Store>
struct PairIO;

template <>
struct PairIO<float> {
  using Word = float2;
  __device__ __forceinline__ static F2 to_f2(Word w) { return F2(w); }
  __device__ __forceinline__ static F2 straddle(Word lo, Word hi) { return F2(lo.y, hi.x); }
  __device__ __forceinline__ static Word from_f2(F2 v) { return v.v; }
};

template <>
struct PairIO<__half> {
  using Word = unsigned;
  __device__ __forceinline__ static F2 to_f2(Word w) {
    __half2 h;
    *reinterpret_cast<unsigned*>(&h) = w;
    return F2(__half22float2(h));
  }
  __device__ __forceinline__ static F2 straddle(Word lo, Word hi) { return to_f2(__byte_perm(lo, hi, 0x5432)); }
  __device__ __forceinline__ static Word from_f2(F2 v) {
    const __half2 h = __float22half2_rn(v.v);
    return *reinterpret_cast<const unsigned*>(&h);
  }
};

template <>
struct PairIO<__nv_bfloat16> {
  using Word = unsigned;
  __device__ __forceinline__ static F2 to_f2(Word w) {
    // a BF16 value is the upper half of the FP32 with the same bits
    return F2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
  }
  __device__ __forceinline__ static F2 straddle(Word lo, Word hi) { return to_f2(__byte_perm(lo, hi, 0x5432)); }
  __device__ __forceinline__ static Word from_f2(F2 v) {
    const __nv_bfloat162 h = __float22bfloat162_rn(v.v);
    return *reinterpret_cast<const unsigned*>(&h);
  }
};

// The 41 populations of the pair (2 i, 2 i + 1) at (y, z) of sublattice s,
// pulled from x - c_q on a periodic grid (the layout of gather(); nx even).
// w: the population array as pair words, (s*41 + q)*n3/2 + ((z*ny + y)*nx)/2 + i.
template <typename Store>
__device__ __forceinline__ void gather_pair(const typename PairIO<Store>::Word* __restrict__ w,
                                            const StepConst<float>& K, int s, int i, int y, int z,
                                            F2 (&h)[kQ]) {
  using IO = PairIO<Store>;
  const int nx = K.nx, ny = K.ny, nz = K.nz, nxp = nx >> 1;
  const int64_t n3p = K.n3 >> 1;
  int yw[5], zw[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    yw[k] = wrap_near(y + k - 2, ny);
    zw[k] = wrap_near(z + k - 2, nz);
  }
  // pair columns i - 1, i, i + 1
  const int ip[3] = {i == 0 ? nxp - 1 : i - 1, i, i == nxp - 1 ? 0 : i + 1};
  // half-velocity sources: c > 0 -> index - 1 on sublattice 0 (else the same),
  // c < 0 -> index + 1 on sublattice 1 (else the same)
  const int yhp = s ? yw[2] : yw[1], yhm = s ? yw[3] : yw[2];
  const int zhp = s ? zw[2] : zw[1], zhm = s ? zw[3] : zw[2];
  const typename IO::Word* same = w + (int64_t)(s * kQ) * n3p;
  const typename IO::Word* other = w + (int64_t)((1 - s) * kQ) * n3p;
  h[0] = IO::to_f2(same[(((int64_t)z * ny + y) * nx >> 1) + i]);
  static_for<kQ - 1>([&](auto qc) {
    constexpr int q = decltype(qc)::value + 1;
    constexpr Vel2 v = vel2(q);
    constexpr bool half = (v.x & 1) != 0;
    int ys, zs;
    const typename IO::Word* base;
    if constexpr (half) {
      ys = v.y > 0 ? yhp : yhm;
      zs = v.z > 0 ? zhp : zhm;
      base = other;
    } else {
      ys = yw[2 - v.y / 2];
      zs = zw[2 - v.z / 2];
      base = same;
    }
    const typename IO::Word* row = base + (int64_t)q * n3p + (((int64_t)zs * ny + ys) * nx >> 1);
    if constexpr (half) {
      // x shift 1 (c > 0, s = 0) or -1 (c < 0, s = 1) straddles; otherwise none
      const bool odd = (v.x > 0) == (s == 0);
      if (odd) {
        const int lo = s == 0 ? ip[0] : ip[1];
        h[q] = IO::straddle(row[lo], row[lo + 1 == nxp ? 0 : lo + 1]);
      } else {
        h[q] = IO::to_f2(row[ip[1]]);
      }
    } else if constexpr (v.x == 0) {
      h[q] = IO::to_f2(row[ip[1]]);
    } else if constexpr (v.x == 4 || v.x == -4) {
      // c_x = +-2: the source pair is one column left (+2) or right (-2)
      h[q] = IO::to_f2(row[ip[v.x > 0 ? 0 : 2]]);
    } else {
      // c_x = +-1: straddles columns (i - 1, i) or (i, i + 1)
      h[q] = v.x > 0 ? IO::straddle(row[ip[0]], row[ip[1]]) : IO::straddle(row[ip[1]], row[ip[2]]);
    }
  });
}

}  // namespace rpk

namespace rpk {

// The 41 pair words of the pair (2 i, 2 i + 1), each already the two values of
// the pair (a straddled word is assembled from its two source words); the
// layout and sources of gather_pair. 16-bit storage only.
template <typename Store>
__device__ __forceinline__ void gather_pair_words(const unsigned* __restrict__ w, const StepConst<float>& K,
                                                  int s, int i, int y, int z, unsigned (&hw)[kQ]) {
  static_assert(sizeof(Store) == 2, "pair words of 16-bit storage");
  const int nx = K.nx, ny = K.ny, nz = K.nz, nxp = nx >> 1;
  const int64_t n3p = K.n3 >> 1;
  int yw[5], zw[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    yw[k] = wrap_near(y + k - 2, ny);
    zw[k] = wrap_near(z + k - 2, nz);
  }
  const int ip[3] = {i == 0 ? nxp - 1 : i - 1, i, i == nxp - 1 ? 0 : i + 1};
  const int yhp = s ? yw[2] : yw[1], yhm = s ? yw[3] : yw[2];
  const int zhp = s ? zw[2] : zw[1], zhm = s ? zw[3] : zw[2];
  const unsigned* same = w + (int64_t)(s * kQ) * n3p;
  const unsigned* other = w + (int64_t)((1 - s) * kQ) * n3p;
  auto join = [](unsigned lo, unsigned hi) { return __byte_perm(lo, hi, 0x5432); };
  hw[0] = same[(((int64_t)z * ny + y) * nx >> 1) + i];
  static_for<kQ - 1>([&](auto qc) {
    constexpr int q = decltype(qc)::value + 1;
    constexpr Vel2 v = vel2(q);
    constexpr bool half = (v.x & 1) != 0;
    int ys, zs;
    const unsigned* base;
    if constexpr (half) {
      ys = v.y > 0 ? yhp : yhm;
      zs = v.z > 0 ? zhp : zhm;
      base = other;
    } else {
      ys = yw[2 - v.y / 2];
      zs = zw[2 - v.z / 2];
      base = same;
    }
    const unsigned* row = base + (int64_t)q * n3p + (((int64_t)zs * ny + ys) * nx >> 1);
    if constexpr (half) {
      const bool odd = (v.x > 0) == (s == 0);
      if (odd) {
        const int lo = s == 0 ? ip[0] : ip[1];
        hw[q] = join(row[lo], row[lo + 1 == nxp ? 0 : lo + 1]);
      } else {
        hw[q] = row[ip[1]];
      }
    } else if constexpr (v.x == 0) {
      hw[q] = row[ip[1]];
    } else if constexpr (v.x == 4 || v.x == -4) {
      hw[q] = row[ip[v.x > 0 ? 0 : 2]];
    } else {
      hw[q] = v.x > 0 ? join(row[ip[0]], row[ip[1]]) : join(row[ip[1]], row[ip[2]]);
    }
  });
}

// A pair word as two FP32 values, converted where it is used: the inline
// conversion is not merged with an earlier conversion of the same word, so
// that the word (one register), not its two FP32 values, stays live between
// the moments and the relaxation.
template <typename Store>
__device__ __forceinline__ F2 word_to_f2_here(unsigned w);
template <>
__device__ __forceinline__ F2 word_to_f2_here<__half>(unsigned w) {
  float a, b;
  asm volatile("{\n .reg .b16 lo, hi;\n mov.b32 {lo, hi}, %2;\n cvt.f32.f16 %0, lo;\n cvt.f32.f16 %1, hi;\n}\n"
               : "=f"(a), "=f"(b)
               : "r"(w));
  return F2(a, b);
}

}  // namespace rpk
