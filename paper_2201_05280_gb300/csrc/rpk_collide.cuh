// The fused pull-stream + collide + rotational-exchange kernel (hot path,
// rows a1-a6 of the step; Sec. 5).
#pragma once

#include "rpk_device.cuh"
#include "rpk_pair.cuh"

namespace rpk {

// Collision of one gathered point (or pair of points, V = F2), in place of
// the paper's explicit update (Sec. 5):
//   g' = (1 - 2 beta*) g + 2 beta* f^mix,   in h form: h' = c_keep h + c_relax (f^mix/w - 1)
//   Er' = Er + dt (delta rho/2)(theta - theta_R)/tau1   (rotational exchange)
// hands the 41 relaxed populations to emit(q, value) in the order q = 0, 1, 2,
// ..., returns the moments in m and the exchanged auxiliary rotational energy
// (paper mode: theta_R after the first backward-Euler half step).
// The part after the raw moments: hq(q) gives population q's h for the
// relaxation (the array itself, or a conversion of its stored word).
template <typename Real, bool kPaper = false, typename V, typename HQ, typename Emit>
__device__ __forceinline__ V collide_relax(const StepConst<Real>& K, Mom<V>& m, V e, HQ&& hq, Emit&& emit) {
  recover<Real, kPaper>(m, e, K);
  Herm<V> H;
  mix_coeffs(m, K, H);
  emit(0, fmad(K.c_keep, hq(0), K.c_relax * H.e0));
  static_for<kPairs>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr Vel2 v = kPairVel2[k];
    const V ev = herm_even<v.x, v.y, v.z>(H);
    const V od = herm_odd<v.x, v.y, v.z>(H);
    emit(2 * k + 1, fmad(K.c_keep, hq(2 * k + 1), K.c_relax * (ev + od)));
    emit(2 * k + 2, fmad(K.c_keep, hq(2 * k + 2), K.c_relax * (ev - od)));
  });
  // conservative form: the exchanged auxiliary energy; paper mode: theta_R after
  // the first backward-Euler half step with the time-t theta_T (Sec. 5, step 1)
  if constexpr (kPaper)
    return fmad(K.ra_keep, m.dR, K.ra_t * m.dT);
  else
    return fmad(K.exc * m.rho, m.dth - m.dR, e);
}

template <typename Real, bool kPaper = false, typename V, typename Emit>
__device__ __forceinline__ V collide_emit(const StepConst<Real>& K, const V (&h)[kQ], V e, Emit&& emit,
                                          Mom<V>& m) {
  raw_moments(h, m);
  return collide_relax<Real, kPaper>(K, m, e, [&](int q) { return h[q]; }, emit);
}

// One point: the populations go to out[q * n3].
template <typename Store, typename Real, bool kPaper = false>
__device__ __forceinline__ Real collide_point(const StepConst<Real>& K, const Real (&h)[kQ], Real e,
                                              Store* __restrict__ out, Mom<Real>& m) {
  const int64_t n3 = K.n3;
  return collide_emit<Real, kPaper>(
      K, h, e, [&](int q, Real v) { out[(int64_t)q * n3] = from_real<Store, Real>(v); }, m);
}

// Device status flags: 1 non-finite moment, 2 rho <= 0, 4 theta_T or theta_R <= 0.
template <typename Real>
__device__ __forceinline__ void flag_moments(const Mom<Real>& m, Real theta0,
                                             unsigned* __restrict__ status) {
  const bool ok = (m.rho > Real(0)) && (theta0 + m.dT > Real(0)) && (theta0 + m.dR > Real(0));
  if (!ok) {
    unsigned f = 0;
    if (!(m.rho == m.rho) || !(m.dT == m.dT) || !(m.dR == m.dR)) f |= 1u;
    if (!(m.rho > Real(0))) f |= 2u;
    if (!(theta0 + m.dT > Real(0)) || !(theta0 + m.dR > Real(0))) f |= 4u;
    atomicOr(status, f);
  }
}

// One collision per point after the pull (Sec. 5):
//   g' = (1 - 2 beta*) g + 2 beta* f^mix,   in h form: h' = c_keep h + c_relax (f^mix/w - 1)
//   Er' = Er + dt (delta rho/2)(theta - theta_R)/tau1   (rotational exchange)
// Writes h', e', rho - 1, u (ring slot of this step) and kappa_R.
// FP32/16-bit arithmetic: at most 102 registers, so that five 128-thread blocks
// per SM keep enough loads in flight.
template <typename Store, typename Real, bool kPull, int kBC, bool kPaper>
__global__ void __launch_bounds__(128, sizeof(Real) == 4 ? 5 : 1)
    k_collide(StepConst<Real> K, const Store* __restrict__ pin, Store* __restrict__ pout,
              const Real* __restrict__ e_in, Real* __restrict__ e_out, Real* __restrict__ drho_out,
              Real* __restrict__ u_out, Real* __restrict__ kap_out,
              const Real* __restrict__ ghost, unsigned* __restrict__ status,
              Real* __restrict__ tt_out, const Real* __restrict__ wcol) {
  PointIdx P;
  if (!point_from_block(K, P)) return;
  const int64_t p = (int64_t)P.s * K.n3 + P.cell;
  Real h[kQ];
  gather<Store, Real, kPull, kBC>(pin, ghost, K, P, h, wcol);
  Mom<Real> m;
  const Real es = collide_point<Store, Real, kPaper>(K, h, e_in[p],
                                             pout + (int64_t)(P.s * kQ) * K.n3 + P.cell, m);
  e_out[p] = es;
  drho_out[p] = m.drho;
  const int64_t npts = 2 * K.n3;
  u_out[p] = m.j[0] * m.inv_rho;
  u_out[npts + p] = m.j[1] * m.inv_rho;
  u_out[2 * npts + p] = m.j[2] * m.inv_rho;
  kap_out[p] = K.kapc * m.rho * (K.theta0 + m.dth);
  if constexpr (kPaper) tt_out[p] = m.dT;  // paper mode: theta_T(f) - theta0 of time t
  flag_moments(m, K.theta0, status);
}

}  // namespace rpk

namespace rpk {

// Status flags of two points (as flag_moments).
__device__ __forceinline__ void flag_moments2(const Mom<F2>& m, float theta0, unsigned* __restrict__ status) {
  const float rho[2] = {m.rho.v.x, m.rho.v.y}, dT[2] = {m.dT.v.x, m.dT.v.y}, dR[2] = {m.dR.v.x, m.dR.v.y};
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const bool ok = (rho[l] > 0.0f) && (theta0 + dT[l] > 0.0f) && (theta0 + dR[l] > 0.0f);
    if (!ok) {
      unsigned f = 0;
      if (!(rho[l] == rho[l]) || !(dT[l] == dT[l]) || !(dR[l] == dR[l])) f |= 1u;
      if (!(rho[l] > 0.0f)) f |= 2u;
      if (!(theta0 + dT[l] > 0.0f) || !(theta0 + dR[l] > 0.0f)) f |= 4u;
      atomicOr(status, f);
    }
  }
}

// The pull-stream + collide + exchange step of k_collide for two x-adjacent
// points per thread on a periodic grid with nx even, FP32 arithmetic in
// packed FP32x2 form (the one-point kernel's FP32 arithmetic to rounding, half
// the arithmetic instructions; pair words halve the loads and stores).
// Thread (blockIdx.x * blockDim.x + threadIdx.x) owns x0 = 2 * that index.
// kPaper: the paper's theta_R solver (the state holds theta_R - theta0; the
// time-t theta_T(f) - theta0 goes to tt_out), as in k_collide.
template <typename Store, bool kPaper = false>
__global__ void __launch_bounds__(128, sizeof(Store) == 4 ? 3 : 4)
    k_collide_pair(StepConst<float> K, const Store* __restrict__ pin, Store* __restrict__ pout,
                   const float* __restrict__ e_in, float* __restrict__ e_out, float* __restrict__ drho_out,
                   float* __restrict__ u_out, float* __restrict__ kap_out, unsigned* __restrict__ status,
                   float* __restrict__ tt_out) {
  using IO = PairIO<Store>;
  using Word = typename IO::Word;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (K.nx >> 1)) return;
  const int y = blockIdx.y;
  const int s = blockIdx.z / K.nz;
  const int z = blockIdx.z - s * K.nz;
  const int64_t n3p = K.n3 >> 1;                                     // pairs per sublattice
  const int64_t cellp = ((((int64_t)z * K.ny + y) * K.nx) >> 1) + i;  // pair of the cell
  const int64_t pp = (int64_t)s * n3p + cellp;                        // pair in a field plane
  F2 h[kQ];
  gather_pair<Store>(reinterpret_cast<const Word*>(pin), K, s, i, y, z, h);
  Mom<F2> m;
  Word* out = reinterpret_cast<Word*>(pout) + (int64_t)(s * kQ) * n3p + cellp;
  const F2 es = collide_emit<float, kPaper>(
      K, h, F2(reinterpret_cast<const float2*>(e_in)[pp]),
      [&](int q, F2 v) { out[(int64_t)q * n3p] = IO::from_f2(v); }, m);
  reinterpret_cast<float2*>(e_out)[pp] = es.v;
  reinterpret_cast<float2*>(drho_out)[pp] = m.drho.v;
  float2* u2 = reinterpret_cast<float2*>(u_out);
  u2[pp] = (m.j[0] * m.inv_rho).v;
  u2[K.n3 + pp] = (m.j[1] * m.inv_rho).v;
  u2[2 * K.n3 + pp] = (m.j[2] * m.inv_rho).v;
  reinterpret_cast<float2*>(kap_out)[pp] = (K.kapc * m.rho * (K.theta0 + m.dth)).v;
  if constexpr (kPaper) reinterpret_cast<float2*>(tt_out)[pp] = m.dT.v;
  flag_moments2(m, K.theta0, status);
}

// FP16 storage: k_collide_pair holding the 41 pair words (one register
// each) instead of their 82 FP32 values between the moments and the
// relaxation, which converts each word again where it is used (one cvt per
// value). Fewer live registers fit more blocks per SM: per 512^3 launch 10.06
// against 10.46 ms in the conservative form (5 blocks per SM), 10.24 against
// 10.88 ms in the paper's solver (4 blocks; 11.53 ms with 5). BF16 storage
// keeps k_collide_pair (11.18 against 10.13 ms: its conversion is two
// integer operations).
template <typename Store, bool kPaper = false>
__global__ void __launch_bounds__(128, kPaper ? 4 : 5)
    k_collide_pair_w(StepConst<float> K, const Store* __restrict__ pin, Store* __restrict__ pout,
                     const float* __restrict__ e_in, float* __restrict__ e_out, float* __restrict__ drho_out,
                     float* __restrict__ u_out, float* __restrict__ kap_out, unsigned* __restrict__ status,
                     float* __restrict__ tt_out) {
  static_assert(std::is_same<Store, __half>::value, "the word-holding collision serves FP16 storage");
  using IO = PairIO<Store>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (K.nx >> 1)) return;
  const int y = blockIdx.y;
  const int s = blockIdx.z / K.nz;
  const int z = blockIdx.z - s * K.nz;
  const int64_t n3p = K.n3 >> 1;
  const int64_t cellp = ((((int64_t)z * K.ny + y) * K.nx) >> 1) + i;
  const int64_t pp = (int64_t)s * n3p + cellp;
  unsigned hw[kQ];
  gather_pair_words<Store>(reinterpret_cast<const unsigned*>(pin), K, s, i, y, z, hw);
  Mom<F2> m;
  {
    F2 h[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) h[q] = IO::to_f2(hw[q]);
    raw_moments(h, m);
  }
  unsigned* out = reinterpret_cast<unsigned*>(pout) + (int64_t)(s * kQ) * n3p + cellp;
  const F2 es = collide_relax<float, kPaper>(
      K, m, F2(reinterpret_cast<const float2*>(e_in)[pp]),
      [&](int q) { return word_to_f2_here<Store>(hw[q]); },
      [&](int q, F2 v) { out[(int64_t)q * n3p] = IO::from_f2(v); });
  reinterpret_cast<float2*>(e_out)[pp] = es.v;
  reinterpret_cast<float2*>(drho_out)[pp] = m.drho.v;
  float2* u2 = reinterpret_cast<float2*>(u_out);
  u2[pp] = (m.j[0] * m.inv_rho).v;
  u2[K.n3 + pp] = (m.j[1] * m.inv_rho).v;
  u2[2 * K.n3 + pp] = (m.j[2] * m.inv_rho).v;
  reinterpret_cast<float2*>(kap_out)[pp] = (K.kapc * m.rho * (K.theta0 + m.dth)).v;
  if constexpr (kPaper) reinterpret_cast<float2*>(tt_out)[pp] = m.dT.v;
  flag_moments2(m, K.theta0, status);
}

}  // namespace rpk
