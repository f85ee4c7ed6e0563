// Remaining device kernels of the step and its I/O: rotational transport
// (MacCormack + FTCS), initialisation, reservoir table, moments and FP64
// diagnostics (Sec. 4 and Sec. 5 of arXiv 2201.05280).
#pragma once

#include "rpk_collide.cuh"

namespace rpk {

// Point of a (32 x 8) thread block of the transport passes: threadIdx.x runs
// along x and threadIdx.y along y, so the y neighbours of most threads are
// loaded by the same block and served from L1.
constexpr int kTBX = 32, kTBY = 8;

template <typename Real>
__device__ __forceinline__ bool point_from_block2d(const StepConst<Real>& K, PointIdx& P) {
  P.x = blockIdx.x * kTBX + threadIdx.x;
  P.y = blockIdx.y * kTBY + threadIdx.y;
  P.s = blockIdx.z / K.nz;
  P.z = blockIdx.z - P.s * K.nz;
  if (P.x >= K.nx || P.y >= K.ny) return false;
  P.cell = ((int64_t)P.z * K.ny + P.y) * K.nx + P.x;
  return true;
}

// Axis neighbour on the same sublattice, or -1 / -2 for the low / high x
// reservoir (kBC == 1), -3 / -4 for the low / high y wall (kBC & kWallY),
// -5 / -6 for the low / high x wall (kBC & kWallX).
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
    if (kBC & kWallX) {
      if (x < 0) return -5;
      if (x >= K.nx) return -6;
    }
    x = wrap_near(x, K.nx);
  } else if (axis == 1) {
    y += d;
    if (kBC & kWallY) {
      if (y < 0) return -3;
      if (y >= K.ny) return -4;
    }
    y = wrap_near(y, K.ny);
  } else {
    z = wrap_near(z + d, K.nz);
  }
  return (int64_t)P.s * K.n3 + ((int64_t)z * K.ny + y) * K.nx + x;
}

// The six axis neighbours of a point as element offsets from the point (the
// periodic wrap folded in), computed once per thread, and the ghost code of a
// neighbour that lies beyond a reservoir or a wall (0 inside; else the
// negative code of axis_nb). Same neighbours as axis_nb, without recomputing a
// 64-bit index per neighbour.
struct NbOff {
  int64_t o[3][2];  // [axis][d = -1, +1]
};

template <typename Real>
__device__ __forceinline__ NbOff nb_offsets(const StepConst<Real>& K, const PointIdx& P) {
  NbOff n;
  const int64_t pl = (int64_t)K.nx * K.ny;
  n.o[0][0] = P.x > 0 ? -1 : K.nx - 1;
  n.o[0][1] = P.x < K.nx - 1 ? 1 : 1 - K.nx;
  n.o[1][0] = P.y > 0 ? -(int64_t)K.nx : (int64_t)(K.ny - 1) * K.nx;
  n.o[1][1] = P.y < K.ny - 1 ? (int64_t)K.nx : -(int64_t)(K.ny - 1) * K.nx;
  n.o[2][0] = P.z > 0 ? -pl : (int64_t)(K.nz - 1) * pl;
  n.o[2][1] = P.z < K.nz - 1 ? pl : -(int64_t)(K.nz - 1) * pl;
  return n;
}

template <int kBC, typename Real>
__device__ __forceinline__ int ghost_code(const StepConst<Real>& K, const PointIdx& P, int a, int d) {
  if (a == 0 && (kBC == 1 || (kBC & kWallX))) {
    if (d < 0 && P.x == 0) return kBC == 1 ? -1 : -5;
    if (d > 0 && P.x == K.nx - 1) return kBC == 1 ? -2 : -6;
  }
  if (a == 1 && (kBC & kWallY)) {
    if (d < 0 && P.y == 0) return -3;
    if (d > 0 && P.y == K.ny - 1) return -4;
  }
  return 0;
}

// Ghost block of a negative axis_nb result: -1, -3 -> 0; -2, -4 -> 1; -5 -> 2; -6 -> 3.
template <typename Real>
__device__ __forceinline__ const Real* ghost_block(const Real* __restrict__ ghost, int64_t q) {
  const int b = q >= -4 ? (int)((-1 - q) & 1) : (int)(-3 - q);
  return ghost + b * kGhostStride;
}

// Wall ghost of theta_R - theta0 for the diffusion: the face flux to the wall
// is kappa_R(p)(theta_w - theta_R(p))/d, d the distance from the point to the
// wall (1/4 for sublattice 0 at a low wall and sublattice 1 at a high wall,
// 3/4 otherwise), written as the value theta_w + (theta_w - theta_p)(1 - d)/d
// on the axis neighbour (whose face coefficient is then kappa_R(p)).
template <typename Real>
__device__ __forceinline__ Real wall_line(Real thw, int64_t q, int s, Real thp) {
  const bool low = (q == -3 || q == -5);
  const Real r = (low == (s == 0)) ? Real(3) : Real(1.0 / 3.0);
  return thw + (thw - thp) * r;
}

template <typename Real>
__device__ __forceinline__ Real wall_theta(const StepConst<Real>& K, const Real* __restrict__ g,
                                           int64_t q, int s, Real thp) {
  const Real thw = (Real(2) * g[kGhE] - K.delta * K.theta0 * g[kGhDrho]) /
                   (K.delta * (Real(1) + g[kGhDrho]));
  return wall_line(thw, q, s, thp);
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
  const NbOff no = nb_offsets(K, P);
  Real acc = Real(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int d = -1; d <= 1; d += 2) {
      const int gc = ghost_code<kBC>(K, P, a, d);
      const int64_t q = gc < 0 ? (int64_t)gc : p + no.o[a][(d + 1) / 2];
      Real thq, kq;
      if (kBC == 1 && q < 0) {
        const Real* g = ghost_block(ghost, q);
        thq = dthR(g[kGhE], g[kGhDrho]);
        kq = g[kGhKap];
      } else if ((kBC & (kWallX | kWallY)) && q < 0) {
        thq = wall_theta(K, ghost_block(ghost, q), q, P.s, th);
        kq = kp;
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
// Rotational transport in three bandwidth-bound passes over the grid:
//   k_mac_pred   MacCormack predictor (forward differences) in flux form
//                F = Er v, with the advecting velocity v = (3 u(t) - u(t-1))/2;
//                also stores v for the corrector
//   k_mac_corr   corrector (backward differences): Er' = (Er + Er_p - dt div F_p)/2;
//                also stores theta_R - theta0 of the result for the diffusion
//   k_ftcs_first first FTCS sub-step of dEr/dt = div(kappa_R grad theta_R) from the
//                stored theta_R (no division per neighbour)
// Further sub-steps use k_ftcs. Reservoir values stand beyond the x ends.
template <typename Real, int kBC>
__global__ void __launch_bounds__(kTBX * kTBY)
    k_mac_pred(StepConst<Real> K, const Real* __restrict__ e, const Real* __restrict__ ucur,
               const Real* __restrict__ uprev, Real* __restrict__ ep, Real* __restrict__ v,
               const Real* __restrict__ ghost) {
  PointIdx P;
  if (!point_from_block2d(K, P)) return;
  const int64_t npts = 2 * K.n3;
  const int64_t p = (int64_t)P.s * K.n3 + P.cell;
  const NbOff no = nb_offsets(K, P);
  const Real ep0 = e[p];
  Real div = Real(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Real vp = vadv(ucur, uprev, a * npts + p);
    v[a * npts + p] = vp;
    const int gc = ghost_code<kBC>(K, P, a, +1);
    const int64_t q = gc < 0 ? (int64_t)gc : p + no.o[a][1];
    Real eq, vq;
    if (kBC != 0 && q < 0) {
      const Real* g = ghost_block(ghost, q);  // a wall has zero normal velocity: no flux
      eq = g[kGhE];
      vq = g[kGhU + a];
    } else {
      eq = e[q];
      vq = vadv(ucur, uprev, a * npts + q);
    }
    div += K.E0 * (vq - vp) + (eq * vq - ep0 * vp);
  }
  ep[p] = ep0 - K.dt * div;
}

template <typename Real, int kBC>
__global__ void __launch_bounds__(kTBX * kTBY)
    k_mac_corr(StepConst<Real> K, const Real* __restrict__ e, const Real* __restrict__ ep,
               const Real* __restrict__ v, const Real* __restrict__ drho, Real* __restrict__ ec,
               Real* __restrict__ th, const Real* __restrict__ ghost) {
  PointIdx P;
  if (!point_from_block2d(K, P)) return;
  const int64_t npts = 2 * K.n3;
  const int64_t p = (int64_t)P.s * K.n3 + P.cell;
  const NbOff no = nb_offsets(K, P);
  const Real epp = ep[p];
  Real div = Real(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Real vp = v[a * npts + p];
    const int gc = ghost_code<kBC>(K, P, a, -1);
    const int64_t q = gc < 0 ? (int64_t)gc : p + no.o[a][0];
    Real eq, vq;
    if (kBC != 0 && q < 0) {
      const Real* g = ghost_block(ghost, q);  // a wall has zero normal velocity: no flux
      eq = g[kGhE];
      vq = g[kGhU + a];
    } else {
      eq = ep[q];
      vq = v[a * npts + q];
    }
    div += K.E0 * (vp - vq) + (epp * vp - eq * vq);
  }
  const Real val = Real(0.5) * (e[p] + epp - K.dt * div);
  const Real dr = drho[p];
  ec[p] = val;
  th[p] = (Real(2) * val - K.delta * K.theta0 * dr) / (K.delta * (Real(1) + dr));
}

template <typename Real, int kBC>
__global__ void __launch_bounds__(kTBX * kTBY)
    k_ftcs_first(StepConst<Real> K, const Real* __restrict__ ec, const Real* __restrict__ th,
                 const Real* __restrict__ kap, Real* __restrict__ e_next,
                 const Real* __restrict__ ghost) {
  PointIdx P;
  if (!point_from_block2d(K, P)) return;
  const int64_t p = (int64_t)P.s * K.n3 + P.cell;
  const Real t0d = K.delta * K.theta0;
  const Real thp = th[p];
  const Real kp = kap[p];
  const NbOff no = nb_offsets(K, P);
  Real acc = Real(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int d = -1; d <= 1; d += 2) {
      const int gc = ghost_code<kBC>(K, P, a, d);
      const int64_t q = gc < 0 ? (int64_t)gc : p + no.o[a][(d + 1) / 2];
      Real thq, kq;
      if (kBC == 1 && q < 0) {
        const Real* g = ghost_block(ghost, q);
        thq = (Real(2) * g[kGhE] - t0d * g[kGhDrho]) / (K.delta * (Real(1) + g[kGhDrho]));
        kq = g[kGhKap];
      } else if ((kBC & (kWallX | kWallY)) && q < 0) {
        thq = wall_theta(K, ghost_block(ghost, q), q, P.s, thp);
        kq = kp;
      } else {
        thq = th[q];
        kq = kap[q];
      }
      acc += Real(0.5) * (kp + kq) * (thq - thp);
    }
  }
  e_next[p] = ec[p] + K.hsub * acc;
}

// ---------------------------------------------------------------------------
// The same three transport passes on a periodic FP32 grid with nx a multiple
// of 4, four x-adjacent points per thread: every field is read and written as
// aligned 16-byte quads, the y and z neighbours of a quad are quads too, and
// only the x neighbours beyond the quad's ends (x0 - 1, x0 + 4) are single
// values. Same expressions in the same order as k_mac_pred, k_mac_corr and
// k_ftcs_first (identical results), four times the bytes in flight per
// thread. Block (32, 8): threadIdx.x runs over quads along x.
struct Quad {
  int x0, y, z, s;
  int64_t p;             // element index of the quad's first point
  int64_t xm, xp;        // offsets of x0 - 1 and x0 + 4 from p (periodic)
  int64_t ym, yp, zm, zp;  // offsets of the neighbour rows / planes
};

inline __device__ bool quad_from_block(const StepConst<float>& K, Quad& Q) {
  Q.x0 = 4 * (blockIdx.x * kTBX + threadIdx.x);
  Q.y = blockIdx.y * kTBY + threadIdx.y;
  Q.s = blockIdx.z / K.nz;
  Q.z = blockIdx.z - Q.s * K.nz;
  if (Q.x0 >= K.nx || Q.y >= K.ny) return false;
  const int64_t pl = (int64_t)K.nx * K.ny;
  Q.p = (int64_t)Q.s * K.n3 + ((int64_t)Q.z * K.ny + Q.y) * K.nx + Q.x0;
  Q.xm = Q.x0 > 0 ? -1 : K.nx - 1;
  Q.xp = Q.x0 + 4 < K.nx ? 4 : 4 - K.nx;
  Q.ym = Q.y > 0 ? -(int64_t)K.nx : (int64_t)(K.ny - 1) * K.nx;
  Q.yp = Q.y < K.ny - 1 ? (int64_t)K.nx : -(int64_t)(K.ny - 1) * K.nx;
  Q.zm = Q.z > 0 ? -pl : (int64_t)(K.nz - 1) * pl;
  Q.zp = Q.z < K.nz - 1 ? pl : -(int64_t)(K.nz - 1) * pl;
  return true;
}

__device__ __forceinline__ float4 ld4(const float* __restrict__ a, int64_t i) {
  return *reinterpret_cast<const float4*>(a + i);
}
__device__ __forceinline__ void st4(float* __restrict__ a, int64_t i, const float (&v)[4]) {
  *reinterpret_cast<float4*>(a + i) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void un4(float4 q, float (&v)[4]) {
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}

static __global__ void __launch_bounds__(kTBX * kTBY)
    k_mac_pred4(StepConst<float> K, const float* __restrict__ e, const float* __restrict__ ucur,
                const float* __restrict__ uprev, float* __restrict__ ep, float* __restrict__ v) {
  Quad Q;
  if (!quad_from_block(K, Q)) return;
  const int64_t npts = 2 * K.n3, p = Q.p;
  float e0[4], div[4] = {0.f, 0.f, 0.f, 0.f}, vp[3][4];
  un4(ld4(e, p), e0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float uc[4], up[4];
    un4(ld4(ucur, a * npts + p), uc);
    un4(ld4(uprev, a * npts + p), up);
#pragma unroll
    for (int l = 0; l < 4; ++l) vp[a][l] = 1.5f * uc[l] - 0.5f * up[l];
    // forward neighbours of the four points along axis a
    float eq[4], vq[4];
    if (a == 0) {
#pragma unroll
      for (int l = 0; l < 3; ++l) eq[l] = e0[l + 1];
      eq[3] = e[p + Q.xp];
      for (int l = 0; l < 3; ++l) vq[l] = vp[0][l + 1];
      vq[3] = vadv(ucur, uprev, p + Q.xp);
    } else {
      const int64_t o = a == 1 ? Q.yp : Q.zp;
      float uq[4], upq[4];
      un4(ld4(e, p + o), eq);
      un4(ld4(ucur, a * npts + p + o), uq);
      un4(ld4(uprev, a * npts + p + o), upq);
#pragma unroll
      for (int l = 0; l < 4; ++l) vq[l] = 1.5f * uq[l] - 0.5f * upq[l];
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) div[l] += K.E0 * (vq[l] - vp[a][l]) + (eq[l] * vq[l] - e0[l] * vp[a][l]);
    st4(v, a * npts + p, vp[a]);
  }
  float r[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) r[l] = e0[l] - K.dt * div[l];
  st4(ep, p, r);
}

static __global__ void __launch_bounds__(kTBX * kTBY)
    k_mac_corr4(StepConst<float> K, const float* __restrict__ e, const float* __restrict__ ep,
                const float* __restrict__ v, const float* __restrict__ drho, float* __restrict__ ec,
                float* __restrict__ th) {
  Quad Q;
  if (!quad_from_block(K, Q)) return;
  const int64_t npts = 2 * K.n3, p = Q.p;
  float epp[4], div[4] = {0.f, 0.f, 0.f, 0.f};
  un4(ld4(ep, p), epp);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float vp[4], eq[4], vq[4];
    un4(ld4(v, a * npts + p), vp);
    if (a == 0) {
      eq[0] = ep[p + Q.xm];
      vq[0] = v[p + Q.xm];
#pragma unroll
      for (int l = 1; l < 4; ++l) {
        eq[l] = epp[l - 1];
        vq[l] = vp[l - 1];
      }
    } else {
      const int64_t o = a == 1 ? Q.ym : Q.zm;
      un4(ld4(ep, p + o), eq);
      un4(ld4(v, a * npts + p + o), vq);
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) div[l] += K.E0 * (vp[l] - vq[l]) + (epp[l] * vp[l] - eq[l] * vq[l]);
  }
  float e0[4], dr[4], val[4], t[4];
  un4(ld4(e, p), e0);
  un4(ld4(drho, p), dr);
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    val[l] = 0.5f * (e0[l] + epp[l] - K.dt * div[l]);
    t[l] = (2.f * val[l] - K.delta * K.theta0 * dr[l]) / (K.delta * (1.f + dr[l]));
  }
  st4(ec, p, val);
  st4(th, p, t);
}

static __global__ void __launch_bounds__(kTBX * kTBY)
    k_ftcs_first4(StepConst<float> K, const float* __restrict__ ec, const float* __restrict__ th,
                  const float* __restrict__ kap, float* __restrict__ e_next) {
  Quad Q;
  if (!quad_from_block(K, Q)) return;
  const int64_t p = Q.p;
  float thp[4], kp[4], acc[4] = {0.f, 0.f, 0.f, 0.f};
  un4(ld4(th, p), thp);
  un4(ld4(kap, p), kp);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int d = -1; d <= 1; d += 2) {
      float thq[4], kq[4];
      if (a == 0) {
        if (d < 0) {
          thq[0] = th[p + Q.xm];
          kq[0] = kap[p + Q.xm];
#pragma unroll
          for (int l = 1; l < 4; ++l) {
            thq[l] = thp[l - 1];
            kq[l] = kp[l - 1];
          }
        } else {
#pragma unroll
          for (int l = 0; l < 3; ++l) {
            thq[l] = thp[l + 1];
            kq[l] = kp[l + 1];
          }
          thq[3] = th[p + Q.xp];
          kq[3] = kap[p + Q.xp];
        }
      } else {
        const int64_t o = a == 1 ? (d < 0 ? Q.ym : Q.yp) : (d < 0 ? Q.zm : Q.zp);
        un4(ld4(th, p + o), thq);
        un4(ld4(kap, p + o), kq);
      }
#pragma unroll
      for (int l = 0; l < 4; ++l) acc[l] += 0.5f * (kp[l] + kq[l]) * (thq[l] - thp[l]);
    }
  }
  float c[4], r[4];
  un4(ld4(ec, p), c);
#pragma unroll
  for (int l = 0; l < 4; ++l) r[l] = c[l] + K.hsub * acc[l];
  st4(e_next, p, r);
}

// Paper-mode transport passes with four x-adjacent points per thread (periodic
// FP32 grid, nx a multiple of 4): k_pm_pred, k_pm_corr and k_pm_ftcs point by
// point, in the same order of operations.
static __global__ void __launch_bounds__(kTBX * kTBY)
    k_pm_pred4(StepConst<float> K, const float* __restrict__ r, const float* __restrict__ ucur,
               float* __restrict__ rp) {
  Quad Q;
  if (!quad_from_block(K, Q)) return;
  const int64_t npts = 2 * K.n3, p = Q.p;
  float r0[4], adv[4] = {0.f, 0.f, 0.f, 0.f};
  un4(ld4(r, p), r0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float u[4], rq[4];
    un4(ld4(ucur, a * npts + p), u);
    if (a == 0) {
#pragma unroll
      for (int l = 0; l < 3; ++l) rq[l] = r0[l + 1];
      rq[3] = r[p + Q.xp];
    } else {
      un4(ld4(r, p + (a == 1 ? Q.yp : Q.zp)), rq);
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) adv[l] += u[l] * (rq[l] - r0[l]);
  }
  float o[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) o[l] = r0[l] - K.dt * adv[l];
  st4(rp, p, o);
}

static __global__ void __launch_bounds__(kTBX * kTBY)
    k_pm_corr4(StepConst<float> K, const float* __restrict__ r, const float* __restrict__ rp,
               const float* __restrict__ ucur, float* __restrict__ rc) {
  Quad Q;
  if (!quad_from_block(K, Q)) return;
  const int64_t npts = 2 * K.n3, p = Q.p;
  float q0[4], adv[4] = {0.f, 0.f, 0.f, 0.f};
  un4(ld4(rp, p), q0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float u[4], rq[4];
    un4(ld4(ucur, a * npts + p), u);
    if (a == 0) {
      rq[0] = rp[p + Q.xm];
#pragma unroll
      for (int l = 1; l < 4; ++l) rq[l] = q0[l - 1];
    } else {
      un4(ld4(rp, p + (a == 1 ? Q.ym : Q.zm)), rq);
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) adv[l] += u[l] * (q0[l] - rq[l]);
  }
  float r0[4], o[4];
  un4(ld4(r, p), r0);
#pragma unroll
  for (int l = 0; l < 4; ++l) o[l] = 0.5f * (r0[l] + q0[l] - K.dt * adv[l]);
  st4(rc, p, o);
}

static __global__ void __launch_bounds__(kTBX * kTBY)
    k_pm_ftcs4(StepConst<float> K, const float* __restrict__ r, const float* __restrict__ drho,
               const float* __restrict__ kap, const float* __restrict__ tt, float* __restrict__ rn, int last) {
  Quad Q;
  if (!quad_from_block(K, Q)) return;
  const int64_t p = Q.p;
  float r0[4], lap[4] = {0.f, 0.f, 0.f, 0.f};
  un4(ld4(r, p), r0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float rpl[4], rmi[4];
    if (a == 0) {
#pragma unroll
      for (int l = 0; l < 3; ++l) rpl[l] = r0[l + 1];
      rpl[3] = r[p + Q.xp];
      rmi[0] = r[p + Q.xm];
#pragma unroll
      for (int l = 1; l < 4; ++l) rmi[l] = r0[l - 1];
    } else {
      un4(ld4(r, p + (a == 1 ? Q.yp : Q.zp)), rpl);
      un4(ld4(r, p + (a == 1 ? Q.ym : Q.zm)), rmi);
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) lap[l] += rpl[l] - 2.0f * r0[l] + rmi[l];
  }
  float dr[4], kp[4], o[4];
  un4(ld4(drho, p), dr);
  un4(ld4(kap, p), kp);
#pragma unroll
  for (int l = 0; l < 4; ++l) o[l] = r0[l] + K.hsub * 2.0f * kp[l] / ((1.0f + dr[l]) * K.delta) * lap[l];
  if (last) {
    float t[4];
    un4(ld4(tt, p), t);
#pragma unroll
    for (int l = 0; l < 4; ++l) o[l] = K.ra_keep * o[l] + K.ra_t * t[l];
  }
  st4(rn, p, o);
}

// ---------------------------------------------------------------------------
// Paper mode of the rotational solver (Sec. 5): after the collision has done
// step 1 (first backward-Euler half step, stored in es), three passes on
// theta_R - theta0 with u of time t:
//   k_pm_pred  MacCormack predictor of u . grad theta_R (forward differences)
//   k_pm_corr  corrector (backward differences)
//   k_pm_ftcs  FTCS sub-step of (2/(rho delta)) kappa_R lap theta_R; the last
//              sub-step also applies step 4, the second half step with the
//              stored time-t theta_T
// theta_R - theta0 of the axis neighbour (a, d) in the array r; beyond a
// reservoir its table value, beyond a wall the straight line through the
// wall's theta_R (its table entry holds theta_R - theta0 in this mode) at the
// wall's distance, extrapolated from r at the point itself.
template <typename Real, int kBC>
__device__ __forceinline__ Real pm_nb(const StepConst<Real>& K, const PointIdx& P, const Real* __restrict__ r,
                                      const Real* __restrict__ ghost, int a, int d) {
  const int64_t q = axis_nb<kBC>(K, P, a, d);
  if (kBC == 1 && q < 0) return ghost[(q == -1 ? 0 : kGhostStride) + kGhE];
  if ((kBC & (kWallX | kWallY)) && q < 0)
    return wall_line(ghost_block(ghost, q)[kGhE], q, P.s, r[(int64_t)P.s * K.n3 + P.cell]);
  return r[q];
}

template <typename Real, int kBC>
__global__ void __launch_bounds__(kTBX * kTBY)
    k_pm_pred(StepConst<Real> K, const Real* __restrict__ r, const Real* __restrict__ ucur,
              Real* __restrict__ rp, const Real* __restrict__ ghost) {
  PointIdx P;
  if (!point_from_block2d(K, P)) return;
  const int64_t p = (int64_t)P.s * K.n3 + P.cell, npts = 2 * K.n3;
  const Real r0 = r[p];
  Real adv = Real(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) adv += ucur[a * npts + p] * (pm_nb<Real, kBC>(K, P, r, ghost, a, +1) - r0);
  rp[p] = r0 - K.dt * adv;
}

template <typename Real, int kBC>
__global__ void __launch_bounds__(kTBX * kTBY)
    k_pm_corr(StepConst<Real> K, const Real* __restrict__ r, const Real* __restrict__ rp,
              const Real* __restrict__ ucur, Real* __restrict__ rc, const Real* __restrict__ ghost) {
  PointIdx P;
  if (!point_from_block2d(K, P)) return;
  const int64_t p = (int64_t)P.s * K.n3 + P.cell, npts = 2 * K.n3;
  const Real q0 = rp[p];
  Real adv = Real(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) adv += ucur[a * npts + p] * (q0 - pm_nb<Real, kBC>(K, P, rp, ghost, a, -1));
  rc[p] = Real(0.5) * (r[p] + q0 - K.dt * adv);
}

template <typename Real, int kBC>
__global__ void __launch_bounds__(kTBX * kTBY)
    k_pm_ftcs(StepConst<Real> K, const Real* __restrict__ r, const Real* __restrict__ drho,
              const Real* __restrict__ kap, const Real* __restrict__ tt, Real* __restrict__ rn,
              const Real* __restrict__ ghost, int last) {
  PointIdx P;
  if (!point_from_block2d(K, P)) return;
  const int64_t p = (int64_t)P.s * K.n3 + P.cell;
  const Real r0 = r[p];
  Real lap = Real(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
    lap += pm_nb<Real, kBC>(K, P, r, ghost, a, +1) - Real(2) * r0 + pm_nb<Real, kBC>(K, P, r, ghost, a, -1);
  Real v = r0 + K.hsub * Real(2) * kap[p] / ((Real(1) + drho[p]) * K.delta) * lap;
  if (last) v = K.ra_keep * v + K.ra_t * tt[p];
  rn[p] = v;
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
  // E_R = delta rho theta_R/2 as a deviation from delta theta0/2 (paper mode:
  // the state is theta_R - theta0)
  e = K.paper ? dR
              : Real(0.5) * K.delta * (rho * dR + K.theta0 * drho) -
                    half_dt_over_tau1 * Real(0.5) * K.delta * rho * (dth - dR);
}

// Initial state of every point: writes its own slots (post-stream state), e,
// and u(0) into both ring slots (the first step advects with u(0)). The same
// pass checks the inputs: check[0] receives (as the bits of a non-negative
// double, by atomic maximum) the largest 3 theta_T + delta theta_R, check[1]
// a nonzero word where some rho, theta_T or theta_R is not finite and positive
// or some velocity component is not finite. The inputs may be host memory the
// device can read directly.
template <typename Store, typename Real>
__global__ void __launch_bounds__(128)
    k_init(StepConst<Real> K, Real half_dt_over_tau1, const double* __restrict__ rho_in,
           const double* __restrict__ u_in, const double* __restrict__ T_in,
           const double* __restrict__ R_in, Store* __restrict__ pout, Real* __restrict__ e_out,
           Real* __restrict__ u0, Real* __restrict__ u1, unsigned long long* __restrict__ check) {
  PointIdx P;
  const bool in = point_from_block(K, P);
  double tv = 0.0;
  bool bad = false;
  if (in) {
    const int64_t npts = 2 * K.n3;
    const int64_t p = (int64_t)P.s * K.n3 + P.cell;
    const double r = rho_in[p], T = T_in[p], R = R_in[p];
    const double ux = u_in[p], uy = u_in[npts + p], uz = u_in[2 * npts + p];
    bad = !(r > 0.0) || !(T > 0.0) || !(R > 0.0) || !isfinite(r) || !isfinite(T) || !isfinite(R) ||
          !isfinite(ux) || !isfinite(uy) || !isfinite(uz);
    if (!bad) {
      tv = 3.0 * T + (double)K.delta * R;
      Real h[kQ], e;
      init_point(K, half_dt_over_tau1, r, ux, uy, uz, T, R, h, e);
      Store* out = pout + (int64_t)(P.s * kQ) * K.n3 + P.cell;
#pragma unroll
      for (int q = 0; q < kQ; ++q) out[(int64_t)q * K.n3] = from_real<Store, Real>(h[q]);
      e_out[p] = e;
      u0[p] = Real(ux); u0[npts + p] = Real(uy); u0[2 * npts + p] = Real(uz);
      u1[p] = Real(ux); u1[npts + p] = Real(uy); u1[2 * npts + p] = Real(uz);
    }
  }
  // positive doubles order like their bit patterns: a warp maximum, then one
  // atomic per warp
  unsigned long long bits = (unsigned long long)__double_as_longlong(tv);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = other > bits ? other : bits;
  }
  const unsigned any_bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(check, bits);
    if (any_bad) atomicOr(check + 1, 1ull);
  }
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
              double* __restrict__ T_o, double* __restrict__ R_o, double* __restrict__ E_o,
              const Real* __restrict__ wcol) {
  PointIdx P;
  if (!point_from_block(K, P)) return;
  const int64_t npts = 2 * K.n3;
  const int64_t p = (int64_t)P.s * K.n3 + P.cell;
  Real h[kQ];
  gather<Store, Real, kPull, kBC>(pin, ghost, K, P, h, wcol);
  Mom<Real> m;
  raw_moments(h, m);
  if (K.paper)
    recover<Real, true>(m, e_in[p], K);
  else
    recover<Real, false>(m, e_in[p], K);
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

// Block reduction of the per-thread diagnostics (sums, and the minimum in
// slot 6) into partial[blockIdx.x * kDiagVals + k].
__device__ __forceinline__ void diag_block_reduce(const double (&acc)[kDiagVals - 1],
                                                  double* __restrict__ partial) {
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

template <typename Store, typename Real, bool kPull, int kBC>
__global__ void __launch_bounds__(kDiagThreads, sizeof(Real) == 4 ? 4 : 1)
    k_diag(StepConst<Real> K, const Store* __restrict__ pin, const Real* __restrict__ e_in,
           const Real* __restrict__ ghost, double* __restrict__ partial,
           const Real* __restrict__ wcol) {
  double acc[kDiagVals - 1] = {0, 0, 0, 0, 0, 0, INFINITY};
  const int64_t npts = 2 * K.n3;
  const double t0 = (double)K.theta0;
  [[maybe_unused]] int64_t npts_here = 0;  // points of this thread (FP32 arithmetic)
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npts;
       p += (int64_t)gridDim.x * blockDim.x) {
    PointIdx P;
    P.s = (int)(p / K.n3);
    P.cell = p - (int64_t)P.s * K.n3;
    P.x = (int)(P.cell % K.nx);
    P.y = (int)((P.cell / K.nx) % K.ny);
    P.z = (int)(P.cell / ((int64_t)K.nx * K.ny));
    Real h[kQ];
    gather<Store, Real, kPull, kBC>(pin, ghost, K, P, h, wcol);
    Mom<Real> m;
    raw_moments(h, m);
    double dm, jx, jy, jz, ek, gmin;
    if constexpr (sizeof(Real) == 8) {
      // FP64 path: conserved sums of the stored values, term by term
      dm = kWeightRest * (double)h[0];
      jx = jy = jz = ek = 0.0;
      gmin = kWeightRest * (1.0 + (double)h[0]);
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
    } else {
      // FP32 arithmetic (FP32 or 16-bit storage): the point's sums come from
      // its FP32 moments (deviation form, so they carry the 2^-24 rounding of
      // the deviations, not of rho = 1); FP64 accumulates them across points
      dm = (double)m.drho;
      jx = (double)m.j[0];
      jy = (double)m.j[1];
      jz = (double)m.j[2];
      ek = 0.5 * ((double)m.dP[0] + (double)m.dP[1] + (double)m.dP[2]);
      Real gm = Real(kWeightRest) * (Real(1) + h[0]);
      static_for<kPairs>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const Real w = Real(pair_weight(k));
        gm = fminf(gm, fminf(w * (Real(1) + h[2 * k + 1]), w * (Real(1) + h[2 * k + 2])));
      });
      gmin = (double)gm;
    }
    if (K.paper)
      recover<Real, true>(m, e_in[p], K);
    else
      recover<Real, false>(m, e_in[p], K);
    // paper mode holds theta_R: its energy density delta rho theta_R / 2 (deviation)
    const double Ee = K.paper ? 0.5 * (double)K.delta * ((double)m.rho * ((double)K.theta0 + (double)m.dR) -
                                                          (double)K.theta0)
                              : (double)e_in[p];
    if constexpr (sizeof(Real) == 8) {
      acc[0] += 1.0 + dm;
      // sum g c^2/2 = 3 theta0/2 + sum w h c^2/2 ; Er = delta theta0/2 + e
      acc[4] += (1.5 * t0 + 0.5 * (double)K.delta * t0) + (ek + Ee);
    } else {
      // the per-point constants (1 and 3 theta0/2 + delta theta0/2) are added
      // once per thread below
      acc[0] += dm;
      acc[4] += ek + Ee;
      ++npts_here;
    }
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += jz;
    acc[6] = fmin(acc[6], gmin);
    // H1 from f = (1 - beta*) g + beta* f^mix, per point in the arithmetic
    // precision of the path, accumulated in FP64
    Herm<Real> H;
    mix_coeffs(m, K, H);
    const Real beta = K.beta, keep = Real(1) - K.beta;
    auto hterm = [](Real w, Real fw) {  // w (fw ln fw - fw), fw = f/w
      if constexpr (sizeof(Real) == 8)
        return fw > Real(0) ? w * (fw * log(fw) - fw) : Real(NAN);
      else
        return fw > Real(0) ? w * (fw * __logf(fw) - fw) : Real(NAN);
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
    if constexpr (sizeof(Real) == 8)
      acc[5] += (double)Hp - 0.5 * (double)K.delta * (double)m.rho * log(t0 + (double)m.dR);
    else  // FP32 arithmetic: the rotational term's logarithm in FP32 too
      acc[5] += (double)(Hp - Real(0.5) * K.delta * m.rho * __logf(K.theta0 + m.dR));
  }
  if constexpr (sizeof(Real) == 4) {
    acc[0] += (double)npts_here;
    acc[4] += (double)npts_here * (1.5 * t0 + 0.5 * (double)K.delta * t0);
  }
  diag_block_reduce(acc, partial);
}

// k_diag for two x-adjacent points per thread (periodic pull, FP32
// arithmetic, nx even; kPaper: the state holds theta_R as in the paper's
// solver): the moments and targets in packed FP32x2 form, the logarithms and
// the FP64 accumulation per point. Thread t handles pair t of the field planes
// (sublattice t / (n3/2)).
template <typename Store, bool kPaper>
__global__ void __launch_bounds__(kDiagThreads, 3)
    k_diag_pair(StepConst<float> K, const Store* __restrict__ pin, const float* __restrict__ e_in,
                double* __restrict__ partial) {
  using Word = typename PairIO<Store>::Word;
  double acc[kDiagVals - 1] = {0, 0, 0, 0, 0, 0, INFINITY};
  const int nxp = K.nx >> 1;
  const int64_t n3p = K.n3 >> 1;
  const double t0 = (double)K.theta0;
  int64_t npts_here = 0;
  const float beta = K.beta, keep = 1.f - K.beta;
  auto hterm = [](float w, float fw) {  // w (fw ln fw - fw), fw = f/w
    return fw > 0.f ? w * (fw * __logf(fw) - fw) : NAN;
  };
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 2 * n3p;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / n3p);
    const int64_t cp = t - (int64_t)s * n3p;
    const int i = (int)(cp % nxp);
    const int64_t row = cp / nxp;
    const int y = (int)(row % K.ny), z = (int)(row / K.ny);
    F2 h[kQ];
    gather_pair<Store>(reinterpret_cast<const Word*>(pin), K, s, i, y, z, h);
    Mom<F2> m;
    raw_moments(h, m);
    const F2 e(reinterpret_cast<const float2*>(e_in)[t]);
    recover<float, kPaper>(m, e, K);
    Herm<F2> H;
    mix_coeffs(m, K, H);
    const float w0 = float(kWeightRest);
    const F2 f0 = F2(1.f) + keep * h[0] + beta * H.e0;
    float Hp[2] = {hterm(w0, f0.v.x), hterm(w0, f0.v.y)};
    float gm[2] = {w0 * (1.f + h[0].v.x), w0 * (1.f + h[0].v.y)};
    static_for<kPairs>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr Vel2 v = kPairVel2[k];
      const float w = float(pair_weight(k));
      const F2 ev = herm_even<v.x, v.y, v.z>(H), od = herm_odd<v.x, v.y, v.z>(H);
      const F2 fp = F2(1.f) + keep * h[2 * k + 1] + beta * (ev + od);
      const F2 fm = F2(1.f) + keep * h[2 * k + 2] + beta * (ev - od);
      Hp[0] += hterm(w, fp.v.x) + hterm(w, fm.v.x);
      Hp[1] += hterm(w, fp.v.y) + hterm(w, fm.v.y);
      gm[0] = fminf(gm[0], fminf(w * (1.f + h[2 * k + 1].v.x), w * (1.f + h[2 * k + 2].v.x)));
      gm[1] = fminf(gm[1], fminf(w * (1.f + h[2 * k + 1].v.y), w * (1.f + h[2 * k + 2].v.y)));
    });
    const float drho[2] = {m.drho.v.x, m.drho.v.y}, rho[2] = {m.rho.v.x, m.rho.v.y};
    const float jx[2] = {m.j[0].v.x, m.j[0].v.y}, jy[2] = {m.j[1].v.x, m.j[1].v.y};
    const float jz[2] = {m.j[2].v.x, m.j[2].v.y}, dR[2] = {m.dR.v.x, m.dR.v.y};
    const float ev[2] = {e.v.x, e.v.y};
    const float p0[2] = {m.dP[0].v.x, m.dP[0].v.y}, p1[2] = {m.dP[1].v.x, m.dP[1].v.y};
    const float p2[2] = {m.dP[2].v.x, m.dP[2].v.y};
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      acc[0] += (double)drho[l];
      acc[1] += (double)jx[l];
      acc[2] += (double)jy[l];
      acc[3] += (double)jz[l];
      // paper mode holds theta_R: its energy density delta rho theta_R / 2 (deviation)
      const double Ee = kPaper ? 0.5 * (double)K.delta * ((double)rho[l] * (t0 + (double)dR[l]) - t0)
                               : (double)ev[l];
      acc[4] += 0.5 * ((double)p0[l] + (double)p1[l] + (double)p2[l]) + Ee;
      acc[5] += (double)(Hp[l] - 0.5f * K.delta * rho[l] * __logf(K.theta0 + dR[l]));
      acc[6] = fmin(acc[6], (double)gm[l]);
    }
    npts_here += 2;
  }
  // the per-point constants: 1 (mass) and 3 theta0/2 + delta theta0/2 (energy)
  acc[0] += (double)npts_here;
  acc[4] += (double)npts_here * (1.5 * t0 + 0.5 * (double)K.delta * t0);
  diag_block_reduce(acc, partial);
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

}  // namespace rpk
