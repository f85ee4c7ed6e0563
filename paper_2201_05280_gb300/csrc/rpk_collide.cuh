// The fused pull-stream + collide + rotational-exchange kernel (hot path,
// rows a1-a6 of the step; Sec. 5).
#pragma once

#include "rpk_device.cuh"

namespace rpk {

// One collision per point after the pull (Sec. 5):
//   g' = (1 - 2 beta*) g + 2 beta* f^mix,   in h form: h' = c_keep h + c_relax (f^mix/w - 1)
//   Er' = Er + dt (delta rho/2)(theta - theta_R)/tau1   (rotational exchange)
// Writes h', e', rho - 1, u (ring slot of this step) and kappa_R.
// Collision of one gathered point, in place of the paper's explicit update:
// writes the 41 relaxed populations through `out` (element q at out[q * n3]),
// returns the moments in m and the exchanged auxiliary rotational energy.
template <typename Store, typename Real, bool kPaper = false>
__device__ __forceinline__ Real collide_point(const StepConst<Real>& K, const Real (&h)[kQ], Real e,
                                              Store* __restrict__ out, Mom<Real>& m) {
  raw_moments(h, m);
  recover<Real, kPaper>(m, e, K);
  Herm<Real> H;
  mix_coeffs(m, K, H);
  const int64_t n3 = K.n3;
  out[0] = from_real<Store, Real>(K.c_keep * h[0] + K.c_relax * H.e0);
  static_for<kPairs>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr Vel2 v = kPairVel2[k];
    const Real ev = herm_even<v.x, v.y, v.z>(H);
    const Real od = herm_odd<v.x, v.y, v.z>(H);
    out[(int64_t)(2 * k + 1) * n3] = from_real<Store, Real>(K.c_keep * h[2 * k + 1] + K.c_relax * (ev + od));
    out[(int64_t)(2 * k + 2) * n3] = from_real<Store, Real>(K.c_keep * h[2 * k + 2] + K.c_relax * (ev - od));
  });
  // conservative form: the exchanged auxiliary energy; paper mode: theta_R after
  // the first backward-Euler half step with the time-t theta_T (Sec. 5, step 1)
  if constexpr (kPaper)
    return K.ra_keep * m.dR + K.ra_t * m.dT;
  else
    return e + K.exc * m.rho * (m.dth - m.dR);
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
