// Remaining device kernels of the step and its I/O: rotational transport
// (MacCormack + FTCS), initialisation, reservoir table, moments and FP64
// diagnostics (Sec. 4 and Sec. 5 of arXiv 2201.05280).
#pragma once

#include "rpk_collide.cuh"

namespace rpk {

// Axis neighbour on the same sublattice, or -1 / -2 for the low / high x
// reservoir when kBC == 1.
template <int kBC, typename Real>
__device__ __forceinline__ int64_t axis_nb(const StepConst<Real>& K, const PointIdx& P, int axis,
                                           int d) {
  int x = P.x, y = P.y, z = P.z;
  if (axis == 0) {
    x += d;
    if (kBC == 1) {
      if (x < 0) return -1;
      if (x >= K.nx) return -2;
    }
    x = wrap_near(x, K.nx);
  } else if (axis == 1) {
    y = wrap_near(y + d, K.ny);
  } else {
    z = wrap_near(z + d, K.nz);
  }
  return (int64_t)P.s * K.n3 + ((int64_t)z * K.ny + y) * K.nx + x;
}

// advecting velocity: second-order extrapolation to t + dt/2
template <typename Real>
__device__ __forceinline__ Real vadv(const Real* __restrict__ ucur, const Real* __restrict__ uprev,
                                     int64_t idx) {
  return Real(1.5) * ucur[idx] - Real(0.5) * uprev[idx];
}

// One FTCS sub-step of dEr/dt = div(kappa_R grad theta_R), theta_R = 2 Er/(delta rho),
// face coefficient = mean of the two kappa_R.
template <typename Real, int kBC>
__global__ void __launch_bounds__(128)
    k_ftcs(StepConst<Real> K, const Real* __restrict__ e, const Real* __restrict__ drho,
           const Real* __restrict__ kap, Real* __restrict__ e_next,
           const Real* __restrict__ ghost) {
  PointIdx P;
  if (!point_from_block(K, P)) return;
  const int64_t p = (int64_t)P.s * K.n3 + P.cell;
  const Real t0d = K.delta * K.theta0;
  auto dthR = [&](Real ee, Real dr) { return (Real(2) * ee - t0d * dr) / (K.delta * (Real(1) + dr)); };
  const Real ee = e[p];
  const Real th = dthR(ee, drho[p]);
  const Real kp = kap[p];
  Real acc = Real(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int d = -1; d <= 1; d += 2) {
      const int64_t q = axis_nb<kBC>(K, P, a, d);
      Real thq, kq;
      if (kBC == 1 && q < 0) {
        const Real* g = ghost + (q == -1 ? 0 : kGhostStride);
        thq = dthR(g[kGhE], g[kGhDrho]);
        kq = g[kGhKap];
      } else {
        thq = dthR(e[q], drho[q]);
        kq = kap[q];
      }
      acc += Real(0.5) * (kp + kq) * (thq - th);
    }
  }
  e_next[p] = ee + K.hsub * acc;
}

// ---------------------------------------------------------------------------
// Fused rotational transport: MacCormack predictor, corrector and the first
// FTCS sub-step in one pass (same arithmetic as the unfused scheme:
// forward-difference predictor, backward-difference corrector, one k_ftcs
// sub-step). A block owns a TX x TY tile of x-y cells of one sublattice and
// marches through ZC planes in z. Iteration k stages plane zn = z0 - 2 + k
// (e*, advecting velocity v, rho - 1, kappa_R; tile + halo) into rings of
// shared-memory planes, forms the predictor on plane zn - 1, the corrector
// (with theta_R) on plane zn - 1 and the diffusion update of plane zn - 2. The
// global loads of plane zn + 1 are issued into registers before the compute
// phases of iteration k, so their latency overlaps the arithmetic. Halo cells
// beyond the x ends hold reservoir values.
template <typename Real>
struct TransportTile {
  static constexpr int TX = 32, TY = 8, ZC = 32;
  static constexpr int EX = TX + 4, EY = TY + 4;  // e*, v planes: offsets -2 .. T+1
  static constexpr int PX = TX + 3, PY = TY + 3;  // predictor: offsets -2 .. T
  static constexpr int CX = TX + 2, CY = TY + 2;  // corrector, theta_R, rho, kappa: -1 .. T
  static constexpr int EP = EX * EY, PP = PX * PY, CP = CX * CY;
  static constexpr int kThreads = TX * TY;
  static constexpr int kEPer = (EP + kThreads - 1) / kThreads;  // staged e/v cells per thread
  static constexpr int kCPer = (CP + kThreads - 1) / kThreads;  // staged rho/kappa cells per thread
  // E[3] V[3][3] P[2] C[2] TH[3] D[4] K[4] planes, then x/y wrap tables (ints)
  static constexpr size_t kReals = 3 * EP + 9 * EP + 2 * PP + 2 * CP + 3 * CP + 4 * CP + 4 * CP;
  static constexpr size_t smem_bytes() { return sizeof(Real) * kReals + sizeof(int) * (EX + EY); }
};

__device__ __forceinline__ int wrap_any(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

template <typename Real, int kBC>
__global__ void __launch_bounds__(TransportTile<Real>::kThreads)
    k_transport_fused(StepConst<Real> K, const Real* __restrict__ es,
                      const Real* __restrict__ ucur, const Real* __restrict__ uprev,
                      const Real* __restrict__ drho, const Real* __restrict__ kap,
                      Real* __restrict__ e_out, const Real* __restrict__ ghost) {
  using T = TransportTile<Real>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sE = reinterpret_cast<Real*>(smem_raw);  // [3][EP]
  Real* sV = sE + 3 * T::EP;                     // [3 slots][3 comps][EP]
  Real* sP = sV + 9 * T::EP;                     // [2][PP]
  Real* sC = sP + 2 * T::PP;                     // [2][CP]
  Real* sTH = sC + 2 * T::CP;                    // [3][CP]
  Real* sD = sTH + 3 * T::CP;                    // [4][CP]
  Real* sK = sD + 4 * T::CP;                     // [4][CP]
  int* xw = reinterpret_cast<int*>(sK + 4 * T::CP);  // [EX] wrapped x (or -1/-2 ghost)
  int* yw = xw + T::EX;                               // [EY] wrapped y
  const int nzb = (K.nz + T::ZC - 1) / T::ZC;
  const int s = blockIdx.z / nzb;
  const int x0 = blockIdx.x * T::TX, y0 = blockIdx.y * T::TY, z0 = (blockIdx.z - s * nzb) * T::ZC;
  const int64_t npts = 2 * K.n3;
  const int64_t sbase = (int64_t)s * K.n3;
  const int tid = threadIdx.x;
  const Real t0d = K.delta * K.theta0;
  for (int i = tid; i < T::EX; i += T::kThreads) {
    const int gx = x0 + i - 2;
    xw[i] = (kBC == 1 && gx < 0) ? -1 : (kBC == 1 && gx >= K.nx) ? -2 : wrap_any(gx, K.nx);
  }
  for (int i = tid; i < T::EY; i += T::kThreads) yw[i] = wrap_any(y0 + i - 2, K.ny);
  const Real* gl = ghost;
  const Real* gh = ghost + kGhostStride;
  __syncthreads();

  // registers holding the staged values of one plane
  Real re[T::kEPer], rv0[T::kEPer], rv1[T::kEPer], rv2[T::kEPer];
  Real rd[T::kCPer], rk[T::kCPer];
  auto fetch = [&](int zn) {
    const int zw = wrap_any(zn, K.nz);
#pragma unroll
    for (int j = 0; j < T::kEPer; ++j) {
      const int i = tid + j * T::kThreads;
      if (i < T::EP) {
        const int xv = xw[i % T::EX], ry = i / T::EX;
        if (kBC == 1 && xv < 0) {
          const Real* g = xv == -1 ? gl : gh;
          re[j] = g[kGhE]; rv0[j] = g[kGhU]; rv1[j] = g[kGhU + 1]; rv2[j] = g[kGhU + 2];
        } else {
          const int64_t q = sbase + ((int64_t)zw * K.ny + yw[ry]) * K.nx + xv;
          re[j] = es[q];
          rv0[j] = vadv(ucur, uprev, q);
          rv1[j] = vadv(ucur, uprev, npts + q);
          rv2[j] = vadv(ucur, uprev, 2 * npts + q);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < T::kCPer; ++j) {
      const int i = tid + j * T::kThreads;
      if (i < T::CP) {
        const int cx = i % T::CX, cy = i / T::CX;
        const int xv = xw[cx + 1];
        if (kBC == 1 && xv < 0) {
          const Real* g = xv == -1 ? gl : gh;
          rd[j] = g[kGhDrho]; rk[j] = g[kGhKap];
        } else {
          const int64_t q = sbase + ((int64_t)zw * K.ny + yw[cy + 1]) * K.nx + xv;
          rd[j] = drho[q]; rk[j] = kap[q];
        }
      }
    }
  };
  fetch(z0 - 2);

  for (int k = 0; k < T::ZC + 4; ++k) {
    const int zn = z0 - 2 + k;     // plane staged in this iteration
    const int se = k % 3;          // e/v ring slot of plane zn
    const int sd = k & 3;          // rho/kappa ring slot of plane zn
    __syncthreads();               // previous readers of the slots are done
    // 1. stage plane zn from registers, then issue the loads of plane zn + 1
#pragma unroll
    for (int j = 0; j < T::kEPer; ++j) {
      const int i = tid + j * T::kThreads;
      if (i < T::EP) {
        sE[se * T::EP + i] = re[j];
        sV[(se * 3 + 0) * T::EP + i] = rv0[j];
        sV[(se * 3 + 1) * T::EP + i] = rv1[j];
        sV[(se * 3 + 2) * T::EP + i] = rv2[j];
      }
    }
#pragma unroll
    for (int j = 0; j < T::kCPer; ++j) {
      const int i = tid + j * T::kThreads;
      if (i < T::CP) {
        sD[sd * T::CP + i] = rd[j];
        sK[sd * T::CP + i] = rk[j];
      }
    }
    if (k + 1 < T::ZC + 4) fetch(zn + 1);
    __syncthreads();
    // 2. predictor on plane zn - 1 (forward differences; z neighbour is plane zn)
    if (k >= 1) {
      const int sb = (k + 2) % 3;        // e/v slot of plane zn - 1
      const int sp = (k - 1) & 1;        // predictor slot of plane zn - 1
      for (int i = tid; i < T::PP; i += T::kThreads) {
        const int px = i % T::PX, py = i / T::PX;
        const int r = py * T::EX + px;   // same offsets (-2) in the e plane
        Real val;
        if (kBC == 1 && xw[px] < 0) {
          val = sE[sb * T::EP + r];
        } else {
          const Real e0 = sE[sb * T::EP + r];
          const int rn[3] = {r + 1, r + T::EX, r};
          const int sn[3] = {sb, sb, se};
          Real div = Real(0);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const Real vp = sV[(sb * 3 + a) * T::EP + r];
            const Real vq = sV[(sn[a] * 3 + a) * T::EP + rn[a]];
            const Real eq = sE[sn[a] * T::EP + rn[a]];
            div += K.E0 * (vq - vp) + (eq * vq - e0 * vp);
          }
          val = e0 - K.dt * div;
        }
        sP[sp * T::PP + i] = val;
      }
    }
    __syncthreads();
    // 3. corrector on plane zn - 1 (backward differences; z neighbour is plane
    //    zn - 2), then the theta_R deviation of that plane
    if (k >= 2) {
      const int sb = (k + 2) % 3;        // e/v slot of plane zn - 1
      const int sm = (k + 1) % 3;        // e/v slot of plane zn - 2
      const int pc = (k - 1) & 1;        // predictor of plane zn - 1
      const int pm = k & 1;              // predictor of plane zn - 2
      const int ct = (k - 1) & 1;        // corrector slot of plane zn - 1
      const int sdm = (k + 3) & 3;       // rho/kappa slot of plane zn - 1
      for (int i = tid; i < T::CP; i += T::kThreads) {
        const int cx = i % T::CX, cy = i / T::CX;
        const int r = (cy + 1) * T::EX + (cx + 1);  // e-plane index of this cell
        const int pi = (cy + 1) * T::PX + (cx + 1);  // predictor index of this cell
        Real val;
        if (kBC == 1 && xw[cx + 1] < 0) {
          val = sE[sb * T::EP + r];
        } else {
          const Real epp = sP[pc * T::PP + pi];
          const Real pnb[3] = {sP[pc * T::PP + pi - 1], sP[pc * T::PP + pi - T::PX],
                               sP[pm * T::PP + pi]};
          const int vs[3] = {sb, sb, sm};
          const int vr[3] = {r - 1, r - T::EX, r};
          Real div = Real(0);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const Real vp = sV[(sb * 3 + a) * T::EP + r];
            const Real vq = sV[(vs[a] * 3 + a) * T::EP + vr[a]];
            div += K.E0 * (vp - vq) + (epp * vp - pnb[a] * vq);
          }
          val = Real(0.5) * (sE[sb * T::EP + r] + epp - K.dt * div);
        }
        const Real dr = sD[sdm * T::CP + i];
        sC[ct * T::CP + i] = val;
        sTH[sb * T::CP + i] = (Real(2) * val - t0d * dr) / (K.delta * (Real(1) + dr));
      }
    }
    __syncthreads();
    // 4. first FTCS sub-step on plane zn - 2
    if (k >= 4) {
      const int zo = zn - 2;
      const int s0 = (k + 1) % 3;        // theta slot of plane zn - 2
      const int sl = k % 3;              // plane zn - 3
      const int su = (k + 2) % 3;        // plane zn - 1
      const int k0 = (k + 2) & 3;        // kappa slot of plane zn - 2
      const int kl = (k + 1) & 3;        // plane zn - 3
      const int ku = (k + 3) & 3;        // plane zn - 1
      const int co = k & 1;              // corrector of plane zn - 2
      const int tx = tid % T::TX, ty = tid / T::TX;
      const int x = x0 + tx, y = y0 + ty;
      if (x < K.nx && y < K.ny && zo < K.nz) {
        const int c = (ty + 1) * T::CX + (tx + 1);
        const Real th = sTH[s0 * T::CP + c];
        const Real kc = sK[k0 * T::CP + c];
        // order -x, +x, -y, +y, -z, +z as in k_ftcs
        const int ts[6] = {s0, s0, s0, s0, sl, su};
        const int ks[6] = {k0, k0, k0, k0, kl, ku};
        const int nc[6] = {c - 1, c + 1, c - T::CX, c + T::CX, c, c};
        Real acc = Real(0);
#pragma unroll
        for (int m = 0; m < 6; ++m)
          acc += Real(0.5) * (kc + sK[ks[m] * T::CP + nc[m]]) * (sTH[ts[m] * T::CP + nc[m]] - th);
        e_out[sbase + ((int64_t)zo * K.ny + y) * K.nx + x] = sC[co * T::CP + c] + K.hsub * acc;
      }
    }
  }
}

// Initial state of one point (Sec. 5): f = f^Eq(rho, u, theta_T I),
// g = f - (dt/2) Omega(f) with Omega = (f^Eq(rho, u, theta I) - f)/tau1 (the ES
// term vanishes since sigma = 0), Er = E_R - (dt/2)(delta rho/2)(theta - theta_R)/tau1.
// Outputs h = g/w - 1 and e = Er - delta theta0/2.
template <typename Real>
__device__ __forceinline__ void init_point(const StepConst<Real>& K, Real half_dt_over_tau1,
                                           double rho_d, double ux, double uy, double uz,
                                           double T, double R, Real (&h)[kQ], Real& e) {
  const Real rho = Real(rho_d);
  const Real drho = Real(rho_d - 1.0);
  const Real inv_rho = Real(1) / rho;
  const Real dT = Real(T - (double)K.theta0);
  const Real dR = Real(R - (double)K.theta0);
  const Real dth = (Real(3) * dT + K.delta * dR) * K.inv_3pd;
  const Real j[3] = {rho * Real(ux), rho * Real(uy), rho * Real(uz)};
  Herm<Real> Hf, He;
  const Real Df[6] = {dT, dT, dT, 0, 0, 0};
  const Real De[6] = {dth, dth, dth, 0, 0, 0};
  hermite(drho, rho, inv_rho, j, Df, K.theta0, Hf);
  hermite(drho, rho, inv_rho, j, De, K.theta0, He);
  // g/w - 1 = (f/w - 1) - (dt/(2 tau1)) ((fEq/w - 1) - (f/w - 1))
  h[0] = Hf.e0 - half_dt_over_tau1 * (He.e0 - Hf.e0);
  static_for<kPairs>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr Vel2 v = kPairVel2[k];
    const Real fe = herm_even<v.x, v.y, v.z>(Hf), fo = herm_odd<v.x, v.y, v.z>(Hf);
    const Real ee = herm_even<v.x, v.y, v.z>(He), eo = herm_odd<v.x, v.y, v.z>(He);
    const Real fp = fe + fo, fm = fe - fo, qp = ee + eo, qm = ee - eo;
    h[2 * k + 1] = fp - half_dt_over_tau1 * (qp - fp);
    h[2 * k + 2] = fm - half_dt_over_tau1 * (qm - fm);
  });
  // E_R = delta rho theta_R/2 as a deviation from delta theta0/2
  e = Real(0.5) * K.delta * (rho * dR + K.theta0 * drho) -
      half_dt_over_tau1 * Real(0.5) * K.delta * rho * (dth - dR);
}

// Initial state of every point: writes its own slots (post-stream state), e,
// and u(0) into both ring slots (the first step advects with u(0)).
template <typename Store, typename Real>
__global__ void __launch_bounds__(128)
    k_init(StepConst<Real> K, Real half_dt_over_tau1, const double* __restrict__ rho_in,
           const double* __restrict__ u_in, const double* __restrict__ T_in,
           const double* __restrict__ R_in, Store* __restrict__ pout, Real* __restrict__ e_out,
           Real* __restrict__ u0, Real* __restrict__ u1) {
  PointIdx P;
  if (!point_from_block(K, P)) return;
  const int64_t npts = 2 * K.n3;
  const int64_t p = (int64_t)P.s * K.n3 + P.cell;
  const double ux = u_in[p], uy = u_in[npts + p], uz = u_in[2 * npts + p];
  Real h[kQ], e;
  init_point(K, half_dt_over_tau1, rho_in[p], ux, uy, uz, T_in[p], R_in[p], h, e);
  Store* out = pout + (int64_t)(P.s * kQ) * K.n3 + P.cell;
#pragma unroll
  for (int q = 0; q < kQ; ++q) out[(int64_t)q * K.n3] = from_real<Store, Real>(h[q]);
  e_out[p] = e;
  u0[p] = Real(ux); u0[npts + p] = Real(uy); u0[2 * npts + p] = Real(uz);
  u1[p] = Real(ux); u1[npts + p] = Real(uy); u1[2 * npts + p] = Real(uz);
}

// Reservoir table: for the low (side 0) and high (side 1) x end, the h of the
// equilibrium state (post-collision equals pre-collision there), its e, rho - 1,
// u and kappa_R. states: rho, ux, uy, uz, theta_T, theta_R per side.
template <typename Real>
__global__ void k_ghost(StepConst<Real> K, Real half_dt_over_tau1, const double* __restrict__ st,
                        Real* __restrict__ ghost) {
  const int side = threadIdx.x;
  if (side >= 2) return;
  const double* s = st + 6 * side;
  Real h[kQ], e;
  init_point(K, half_dt_over_tau1, s[0], s[1], s[2], s[3], s[4], s[5], h, e);
  Real* g = ghost + side * kGhostStride;
#pragma unroll
  for (int q = 0; q < kQ; ++q) g[q] = h[q];
  g[kGhE] = e;
  g[kGhDrho] = Real(s[0] - 1.0);
  g[kGhU] = Real(s[1]);
  g[kGhU + 1] = Real(s[2]);
  g[kGhU + 2] = Real(s[3]);
  const double theta = (3.0 * s[4] + (double)K.delta * s[5]) / (3.0 + (double)K.delta);
  g[kGhKap] = Real((double)K.kapc * s[0] * theta);
}

// Hydrodynamic fields of the current state (FP64 outputs).
template <typename Store, typename Real, bool kPull, int kBC>
__global__ void __launch_bounds__(128)
    k_moments(StepConst<Real> K, const Store* __restrict__ pin, const Real* __restrict__ e_in,
              const Real* __restrict__ ghost, double* __restrict__ rho_o, double* __restrict__ u_o,
              double* __restrict__ T_o, double* __restrict__ R_o, double* __restrict__ E_o) {
  PointIdx P;
  if (!point_from_block(K, P)) return;
  const int64_t npts = 2 * K.n3;
  const int64_t p = (int64_t)P.s * K.n3 + P.cell;
  Real h[kQ];
  gather<Store, Real, kPull, kBC>(pin, ghost, K, P, h);
  Mom<Real> m;
  raw_moments(h, m);
  recover(m, e_in[p], K);
  if (rho_o) rho_o[p] = 1.0 + (double)m.drho;
  if (u_o) {
    u_o[p] = (double)(m.j[0] * m.inv_rho);
    u_o[npts + p] = (double)(m.j[1] * m.inv_rho);
    u_o[2 * npts + p] = (double)(m.j[2] * m.inv_rho);
  }
  if (T_o) T_o[p] = (double)K.theta0 + (double)m.dT;
  if (R_o) R_o[p] = (double)K.theta0 + (double)m.dR;
  if (E_o) E_o[p] = 0.5 * (double)K.delta * (1.0 + (double)m.drho) * ((double)K.theta0 + (double)m.dR);
}

// ---- FP64 diagnostics: per-block partial sums, then one block reduces them.
constexpr int kDiagVals = 8;  // M, Jx, Jy, Jz, E, H1, min_g, (unused)
constexpr int kDiagBlocks = 1024;
constexpr int kDiagThreads = 128;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <typename Store, typename Real, bool kPull, int kBC>
__global__ void __launch_bounds__(kDiagThreads)
    k_diag(StepConst<Real> K, const Store* __restrict__ pin, const Real* __restrict__ e_in,
           const Real* __restrict__ ghost, double* __restrict__ partial) {
  double acc[kDiagVals - 1] = {0, 0, 0, 0, 0, 0, INFINITY};
  const int64_t npts = 2 * K.n3;
  const double t0 = (double)K.theta0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npts;
       p += (int64_t)gridDim.x * blockDim.x) {
    PointIdx P;
    P.s = (int)(p / K.n3);
    P.cell = p - (int64_t)P.s * K.n3;
    P.x = (int)(P.cell % K.nx);
    P.y = (int)((P.cell / K.nx) % K.ny);
    P.z = (int)(P.cell / ((int64_t)K.nx * K.ny));
    Real h[kQ];
    gather<Store, Real, kPull, kBC>(pin, ghost, K, P, h);
    // conserved sums in FP64 from the stored values
    double dm = kWeightRest * (double)h[0], jx = 0, jy = 0, jz = 0, ek = 0;
    double gmin = kWeightRest * (1.0 + (double)h[0]);
    static_for<kPairs>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr Vel2 v = kPairVel2[k];
      constexpr double w = pair_weight(k);
      constexpr double c2 = 0.25 * (v.x * v.x + v.y * v.y + v.z * v.z);
      const double hp = (double)h[2 * k + 1], hm = (double)h[2 * k + 2];
      dm += w * (hp + hm);
      jx += 0.5 * v.x * w * (hp - hm);
      jy += 0.5 * v.y * w * (hp - hm);
      jz += 0.5 * v.z * w * (hp - hm);
      ek += 0.5 * c2 * w * (hp + hm);
      gmin = fmin(gmin, fmin(w * (1.0 + hp), w * (1.0 + hm)));
    });
    const double Ee = (double)e_in[p];
    acc[0] += 1.0 + dm;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += jz;
    // sum g c^2/2 = 3 theta0/2 + sum w h c^2/2 ; Er = delta theta0/2 + e
    acc[4] += (1.5 * t0 + 0.5 * (double)K.delta * t0) + (ek + Ee);
    acc[6] = fmin(acc[6], gmin);
    // H1 from f = (1 - beta*) g + beta* f^mix, per point in the arithmetic
    // precision of the path, accumulated in FP64
    Mom<Real> m;
    raw_moments(h, m);
    recover(m, e_in[p], K);
    Herm<Real> H;
    mix_coeffs(m, K, H);
    const Real beta = K.beta, keep = Real(1) - K.beta;
    auto hterm = [](Real w, Real fw) {  // w (fw ln fw - fw), fw = f/w
      return fw > Real(0) ? w * (fw * log(fw) - fw) : Real(NAN);
    };
    Real Hp = hterm(Real(kWeightRest), Real(1) + keep * h[0] + beta * H.e0);
    static_for<kPairs>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr Vel2 v = kPairVel2[k];
      const Real w = Real(pair_weight(k));
      const Real ev = herm_even<v.x, v.y, v.z>(H), od = herm_odd<v.x, v.y, v.z>(H);
      Hp += hterm(w, Real(1) + keep * h[2 * k + 1] + beta * (ev + od));
      Hp += hterm(w, Real(1) + keep * h[2 * k + 2] + beta * (ev - od));
    });
    acc[5] += (double)Hp - 0.5 * (double)K.delta * (double)m.rho * log(t0 + (double)m.dR);
  }
  __shared__ double red[kDiagThreads / 32][kDiagVals];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kDiagVals - 1; ++k) {
    const double v = (k == 6) ? warp_min(acc[k]) : warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kDiagVals - 1) {
    const int k = threadIdx.x;
    double v = red[0][k];
    for (int w = 1; w < kDiagThreads / 32; ++w) v = (k == 6) ? fmin(v, red[w][k]) : v + red[w][k];
    partial[(int64_t)blockIdx.x * kDiagVals + k] = v;
  }
}

static __global__ void __launch_bounds__(1024) k_diag_final(const double* __restrict__ partial, int nblk,
                                                     double* __restrict__ out) {
  __shared__ double red[32][kDiagVals];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < kDiagVals - 1; ++k) {
    double v = (k == 6) ? INFINITY : 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      const double x = partial[(int64_t)b * kDiagVals + k];
      v = (k == 6) ? fmin(v, x) : v + x;
    }
    v = (k == 6) ? warp_min(v) : warp_sum(v);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kDiagVals - 1) {
    const int k = threadIdx.x;
    double v = red[0][k];
    for (int w = 1; w < (int)(blockDim.x / 32); ++w) v = (k == 6) ? fmin(v, red[w][k]) : v + red[w][k];
    out[k] = v;
  }
}

// max over points of theta = (3 theta_T + delta theta_R)/(3 + delta), for nsub
static __global__ void __launch_bounds__(256) k_theta_max(const double* __restrict__ T,
                                                   const double* __restrict__ R, int64_t n,
                                                   double delta, double* __restrict__ out) {
  __shared__ double red[8];
  double v = -INFINITY;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    v = fmax(v, (3.0 * T[p] + delta * R[p]) / (3.0 + delta));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) v = fmax(v, red[w]);
    out[blockIdx.x] = v;
  }
}

}  // namespace rpk
