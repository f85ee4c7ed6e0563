// Kernel launch sequences of one precision (included by rpk_ops_<prec>.cu,
// which instantiate Ops<Store, Real> for their storage type).
#pragma once

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "rpk_internal.h"
#include "rpk_kernels.cuh"

namespace rpk {

// Per-launch constants of the step (Sec. 5) for relaxation parameters r on an
// nx x ny x nz grid with nsub FTCS sub-steps; computed in double, then cast.
template <typename Real>
static StepConst<Real> make_step_const(const rpk_relax& r, int nsub, int nx, int ny, int nz,
                                       int paper = 0) {
  const double tau_s = 1.0 / (1.0 / r.tau + 1.0 / r.tau1);
  const double beta = r.dt / (2.0 * tau_s + r.dt);
  const double B = 1.0 + r.tau / r.tau1;
  StepConst<Real> K;
  K.nx = nx;
  K.ny = ny;
  K.nz = nz;
  K.n3 = (int64_t)nx * ny * nz;
  K.theta0 = Real(kTheta0);
  K.c_keep = Real(1.0 - 2.0 * beta);
  K.c_relax = Real(2.0 * beta);
  K.beta = Real(beta);
  K.w_es = Real(tau_s / r.tau);
  K.w_eq = Real(tau_s / r.tau1);
  K.b = Real(r.b);
  K.inv_sig = Real(1.0 / (1.0 + r.dt / (2.0 * tau_s) - r.b * r.dt / (2.0 * r.tau)));
  K.inv_d = Real(1.0 / (1.0 + r.dt / (2.0 * r.tau1)));
  K.delta = Real(r.delta);
  K.inv_3pd = Real(1.0 / (3.0 + r.delta));
  K.exc = Real(r.dt * r.delta / (2.0 * r.tau1));
  K.kapc = Real(r.k_r * 5.0 * r.tau / (2.0 * B));
  K.E0 = Real(0.5 * r.delta * kTheta0);
  K.dt = Real(r.dt);
  K.hsub = Real(r.dt / std::max(1, nsub));
  const double X = 3.0 * r.dt / (2.0 * r.tau1 * (3.0 + r.delta));
  K.paper = paper;
  K.ra_keep = Real(1.0 / (1.0 + X));
  K.ra_t = Real(X / (1.0 + X));
  K.pa = Real(r.delta * X / 3.0);
  K.inv_1pa = Real(1.0 / (1.0 + r.delta * X / 3.0));
  return K;
}

template <typename Real>
static StepConst<Real> make_const(const rpk_lattice* L) {
  return make_step_const<Real>(L->relax, L->nsub, L->grid.nx, L->grid.ny, L->grid.nz, L->rot_mode);
}

static inline dim3 point_grid(const rpk_lattice* L, int bx) {
  return dim3((unsigned)((L->grid.nx + bx - 1) / bx), (unsigned)L->grid.ny,
              (unsigned)(2 * L->grid.nz));
}

static inline rpk_status check_launch(const char* what) {
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, what);
  return RPK_OK;
}

// Walls in use: kWallY and / or kWallX.
static inline int wall_mask(const rpk_lattice* L) {
  return (L->walls ? kWallY : 0) | (L->xwalls ? kWallX : 0);
}

// rho_w - 1 of every wall column from the current (post-collision)
// populations; precedes every pull when walls are on.
template <typename Store, typename Real, int kBC>
static rpk_status wall_launch_t(rpk_lattice* L, const StepConst<Real>& K) {
  const int64_t n = ((kBC & kWallY) ? 2 * (int64_t)L->grid.nx * L->grid.nz : 0) +
                    ((kBC & kWallX) ? 2 * (int64_t)L->grid.ny * L->grid.nz : 0);
  k_wall_rho<Store, Real, kBC><<<(unsigned)((n + 127) / 128), 128, 0, L->stream>>>(
      K, static_cast<const Store*>(L->pop[L->cur]), static_cast<const Real*>(L->ghost),
      static_cast<Real*>(L->wrho));
  return check_launch("k_wall_rho");
}

template <typename Store, typename Real>
static rpk_status wall_launch(rpk_lattice* L, const StepConst<Real>& K) {
  switch (wall_mask(L)) {
    case kWallY: return wall_launch_t<Store, Real, kWallY>(L, K);
    case kWallX: return wall_launch_t<Store, Real, kWallX>(L, K);
    default: return wall_launch_t<Store, Real, kWallY | kWallX>(L, K);
  }
}

template <typename Store, typename Real, bool kPull, int kBC>
static rpk_status collide_launch(rpk_lattice* L, const StepConst<Real>& K) {
  const Store* pin = static_cast<const Store*>(L->pop[L->cur]);
  Store* pout = static_cast<Store*>(L->pop[L->cur ^ 1]);
  Real* ucur = static_cast<Real*>(L->u[L->steps & 1]);
  const Real* wcol = static_cast<const Real*>(L->wrho);
  if (L->rot_mode) {
    if constexpr (kPull && kBC == 0 && sizeof(Real) == 4) {
      if (L->grid.nx % 2 == 0) {
        // two x-adjacent points per thread, packed FP32x2 arithmetic
        const dim3 grid((unsigned)((L->grid.nx / 2 + 127) / 128), (unsigned)L->grid.ny,
                        (unsigned)(2 * L->grid.nz));
        if constexpr (std::is_same<Store, __half>::value)
          k_collide_pair_w<Store, true><<<grid, 128, 0, L->stream>>>(
              K, pin, pout, static_cast<const Real*>(L->e), static_cast<Real*>(L->e_star),
              static_cast<Real*>(L->drho), ucur, static_cast<Real*>(L->kap), L->status,
              static_cast<Real*>(L->thbuf));
        else
          k_collide_pair<Store, true><<<grid, 128, 0, L->stream>>>(
              K, pin, pout, static_cast<const Real*>(L->e), static_cast<Real*>(L->e_star),
              static_cast<Real*>(L->drho), ucur, static_cast<Real*>(L->kap), L->status,
              static_cast<Real*>(L->thbuf));
        return check_launch("k_collide_pair");
      }
    }
    k_collide<Store, Real, kPull, kBC, true><<<point_grid(L, 128), 128, 0, L->stream>>>(
        K, pin, pout, static_cast<const Real*>(L->e), static_cast<Real*>(L->e_star),
        static_cast<Real*>(L->drho), ucur, static_cast<Real*>(L->kap),
        static_cast<const Real*>(L->ghost), L->status, static_cast<Real*>(L->thbuf), wcol);
    return check_launch("k_collide");
  }
  if constexpr (kPull && kBC == 0 && sizeof(Real) == 4) {
    if (L->grid.nx % 2 == 0) {
      // two x-adjacent points per thread, packed FP32x2 arithmetic
      const dim3 grid((unsigned)((L->grid.nx / 2 + 127) / 128), (unsigned)L->grid.ny,
                      (unsigned)(2 * L->grid.nz));
      // FP16 storage holds the pair words, not their FP32 values, across the collision
      if constexpr (std::is_same<Store, __half>::value)
        k_collide_pair_w<Store, false><<<grid, 128, 0, L->stream>>>(
            K, pin, pout, static_cast<const Real*>(L->e), static_cast<Real*>(L->e_star),
            static_cast<Real*>(L->drho), ucur, static_cast<Real*>(L->kap), L->status, nullptr);
      else
        k_collide_pair<Store, false><<<grid, 128, 0, L->stream>>>(
            K, pin, pout, static_cast<const Real*>(L->e), static_cast<Real*>(L->e_star),
            static_cast<Real*>(L->drho), ucur, static_cast<Real*>(L->kap), L->status, nullptr);
      return check_launch("k_collide_pair");
    }
  }
  k_collide<Store, Real, kPull, kBC, false><<<point_grid(L, 128), 128, 0, L->stream>>>(
      K, pin, pout, static_cast<const Real*>(L->e), static_cast<Real*>(L->e_star),
      static_cast<Real*>(L->drho), ucur, static_cast<Real*>(L->kap),
      static_cast<const Real*>(L->ghost), L->status, nullptr, wcol);
  return check_launch("k_collide");
}

template <typename Real, int kBC>
static rpk_status transport_launch(rpk_lattice* L, const StepConst<Real>& K) {
  const dim3 grid = point_grid(L, 128);
  const Real* ucur = static_cast<const Real*>(L->u[L->steps & 1]);
  const Real* uprev = static_cast<const Real*>(L->u[(L->steps + 1) & 1]);
  const Real* gh = static_cast<const Real*>(L->ghost);
  const Real* drho = static_cast<const Real*>(L->drho);
  const Real* kap = static_cast<const Real*>(L->kap);
  Real* es = static_cast<Real*>(L->e_star);
  Real* ea = static_cast<Real*>(L->e_a);
  Real* eb = static_cast<Real*>(L->e_b);
  Real* v = static_cast<Real*>(L->vbuf);
  Real* th = static_cast<Real*>(L->thbuf);
  Real* e = static_cast<Real*>(L->e);
  const dim3 tb(kTBX, kTBY);
  const dim3 tgrid((unsigned)((L->grid.nx + kTBX - 1) / kTBX),
                   (unsigned)((L->grid.ny + kTBY - 1) / kTBY), (unsigned)(2 * L->grid.nz));
  RPK_CUDA(timing_begin(L));
  if (L->rot_mode) {
    // paper mode: MacCormack on theta_R, FTCS sub-steps, the last with the
    // second relaxation half step (th holds the time-t theta_T)
    if constexpr (kBC == 0 && sizeof(Real) == 4) {
      if (L->grid.nx % 4 == 0) {
        // periodic FP32 grid, nx a multiple of 4: four x-adjacent points per thread
        const dim3 qgrid((unsigned)((L->grid.nx / 4 + kTBX - 1) / kTBX),
                         (unsigned)((L->grid.ny + kTBY - 1) / kTBY), (unsigned)(2 * L->grid.nz));
        k_pm_pred4<<<qgrid, tb, 0, L->stream>>>(K, es, ucur, ea);
        k_pm_corr4<<<qgrid, tb, 0, L->stream>>>(K, es, ea, ucur, eb);
        const Real* src = eb;
        for (int k = 0; k < L->nsub; ++k) {
          Real* dst = (k == L->nsub - 1) ? e : (src == eb ? ea : eb);
          k_pm_ftcs4<<<qgrid, tb, 0, L->stream>>>(K, src, drho, kap, th, dst, k == L->nsub - 1);
          src = dst;
        }
        RPK_CUDA(timing_end(L, RPK_KC_TRANSPORT, 2 + L->nsub));
        return check_launch("rotational transport (paper mode)");
      }
    }
    k_pm_pred<Real, kBC><<<tgrid, tb, 0, L->stream>>>(K, es, ucur, ea, gh);
    k_pm_corr<Real, kBC><<<tgrid, tb, 0, L->stream>>>(K, es, ea, ucur, eb, gh);
    const Real* src = eb;
    for (int k = 0; k < L->nsub; ++k) {
      Real* dst = (k == L->nsub - 1) ? e : (src == eb ? ea : eb);
      k_pm_ftcs<Real, kBC><<<tgrid, tb, 0, L->stream>>>(K, src, drho, kap, th, dst, gh,
                                                         k == L->nsub - 1);
      src = dst;
    }
    RPK_CUDA(timing_end(L, RPK_KC_TRANSPORT, 2 + L->nsub));
    return check_launch("rotational transport (paper mode)");
  }
  // predictor, corrector and the first FTCS sub-step; further sub-steps end in e
  Real* dst = L->nsub == 1 ? e : ea;
  bool quads = false;
  if constexpr (kBC == 0 && sizeof(Real) == 4) quads = L->grid.nx % 4 == 0;
  if (quads) {
    if constexpr (kBC == 0 && sizeof(Real) == 4) {
      // periodic FP32 grid, nx a multiple of 4: four x-adjacent points per thread
      const dim3 qgrid((unsigned)((L->grid.nx / 4 + kTBX - 1) / kTBX),
                       (unsigned)((L->grid.ny + kTBY - 1) / kTBY), (unsigned)(2 * L->grid.nz));
      k_mac_pred4<<<qgrid, tb, 0, L->stream>>>(K, es, ucur, uprev, ea, v);
      k_mac_corr4<<<qgrid, tb, 0, L->stream>>>(K, es, ea, v, drho, eb, th);
      k_ftcs_first4<<<qgrid, tb, 0, L->stream>>>(K, eb, th, kap, dst);
    }
  } else {
    k_mac_pred<Real, kBC><<<tgrid, tb, 0, L->stream>>>(K, es, ucur, uprev, ea, v, gh);
    k_mac_corr<Real, kBC><<<tgrid, tb, 0, L->stream>>>(K, es, ea, v, drho, eb, th, gh);
    k_ftcs_first<Real, kBC><<<tgrid, tb, 0, L->stream>>>(K, eb, th, kap, dst, gh);
  }
  Real* src = dst;
  for (int k = 1; k < L->nsub; ++k) {
    dst = (k == L->nsub - 1) ? e : (src == ea ? eb : ea);
    k_ftcs<Real, kBC><<<grid, 128, 0, L->stream>>>(K, src, drho, kap, dst, gh);
    src = dst;
  }
  RPK_CUDA(timing_end(L, RPK_KC_TRANSPORT, 2 + L->nsub));
  return check_launch("rotational transport");
}

template <typename Store, typename Real>
rpk_status Ops<Store, Real>::step(rpk_lattice* L, int64_t n) {
  const StepConst<Real> K = make_const<Real>(L);
  const bool res = L->grid.bc_x == RPK_BC_RESERVOIR;
  const int wm = wall_mask(L);
  for (int64_t t = 0; t < n; ++t) {
    rpk_status st;
    RPK_CUDA(timing_begin(L));
    const bool wall_pull = wm && !L->streamed;
    if (wall_pull) {
      st = wall_launch<Store, Real>(L, K);
      if (st != RPK_OK) return st;
    }
    if (L->streamed)
      st = res ? collide_launch<Store, Real, false, 1>(L, K) : collide_launch<Store, Real, false, 0>(L, K);
    else if (wm == kWallY)
      st = collide_launch<Store, Real, true, kWallY>(L, K);
    else if (wm == kWallX)
      st = collide_launch<Store, Real, true, kWallX>(L, K);
    else if (wm)
      st = collide_launch<Store, Real, true, kWallY | kWallX>(L, K);
    else
      st = res ? collide_launch<Store, Real, true, 1>(L, K) : collide_launch<Store, Real, true, 0>(L, K);
    if (st != RPK_OK) return st;
    RPK_CUDA(timing_end(L, RPK_KC_COLLIDE, wall_pull ? 2 : 1));
    if (wm == kWallY)
      st = transport_launch<Real, kWallY>(L, K);
    else if (wm == kWallX)
      st = transport_launch<Real, kWallX>(L, K);
    else if (wm)
      st = transport_launch<Real, kWallY | kWallX>(L, K);
    else
      st = res ? transport_launch<Real, 1>(L, K) : transport_launch<Real, 0>(L, K);
    if (st != RPK_OK) return st;
    L->cur ^= 1;
    L->streamed = false;
    L->steps += 1;
  }
  return RPK_OK;
}

template <typename Store, typename Real>
rpk_status Ops<Store, Real>::init(rpk_lattice* L, const double* rho, const double* u,
                                  const double* T, const double* R) {
  const StepConst<Real> K = make_const<Real>(L);
  const Real hdt = Real(0.5 * L->relax.dt / L->relax.tau1);
  L->cur = 0;
  unsigned long long* check = reinterpret_cast<unsigned long long*>(L->diag_out);
  RPK_CUDA(cudaMemsetAsync(check, 0, 2 * sizeof(unsigned long long), L->stream));
  k_init<Store, Real><<<point_grid(L, 128), 128, 0, L->stream>>>(
      K, hdt, rho, u, T, R, static_cast<Store*>(L->pop[0]), static_cast<Real*>(L->e),
      static_cast<Real*>(L->u[0]), static_cast<Real*>(L->u[1]), check);
  return check_launch("k_init");
}

template <typename Store, typename Real>
rpk_status Ops<Store, Real>::ghosts(rpk_lattice* L) {
  const StepConst<Real> K = make_const<Real>(L);
  const Real hdt = Real(0.5 * L->relax.dt / L->relax.tau1);
  double* dst = L->diag_partial;  // 24 doubles of staging
  // blocks 0, 1: the reservoirs' states or the y walls; blocks 2, 3: the x
  // walls. A wall's state: rho = 1 at its velocity, theta_T = theta_R = theta_w.
  double st24[24] = {0};
  auto wall_state = [&](const double* wl, double* out6) {
    const double s6[6] = {1.0, wl[0], wl[1], wl[2], wl[3], wl[3]};
    for (int k = 0; k < 6; ++k) out6[k] = s6[k];
  };
  const double rest[4] = {0.0, 0.0, 0.0, kTheta0};  // fills blocks nothing reads
  if (L->walls) {
    wall_state(L->wall, st24);
    wall_state(L->wall + 4, st24 + 6);
  } else if (L->grid.bc_x == RPK_BC_RESERVOIR) {
    for (int k = 0; k < 12; ++k) st24[k] = L->res[k];
  } else {
    wall_state(rest, st24);
    wall_state(rest, st24 + 6);
  }
  wall_state(L->xwalls ? L->xwall : rest, st24 + 12);
  wall_state(L->xwalls ? L->xwall + 4 : rest, st24 + 18);
  RPK_CUDA(cudaMemcpyAsync(dst, st24, 24 * sizeof(double), cudaMemcpyHostToDevice, L->stream));
  k_ghost<Real><<<1, 32, 0, L->stream>>>(K, hdt, dst, static_cast<Real*>(L->ghost));
  rpk_status st = check_launch("k_ghost");
  if (st != RPK_OK) return st;
  k_ghost<Real><<<1, 32, 0, L->stream>>>(K, hdt, dst + 12, static_cast<Real*>(L->ghost) + 2 * kGhostStride);
  st = check_launch("k_ghost");
  if (st != RPK_OK) return st;
  RPK_CUDA(cudaStreamSynchronize(L->stream));
  return RPK_OK;
}

template <typename Store, typename Real>
rpk_status Ops<Store, Real>::moments(rpk_lattice* L, double* rho, double* u, double* T,
                                     double* R, double* E) {
  const StepConst<Real> K = make_const<Real>(L);
  const Store* pin = static_cast<const Store*>(L->pop[L->cur]);
  const Real* e = static_cast<const Real*>(L->e);
  const Real* gh = static_cast<const Real*>(L->ghost);
  const Real* wcol = static_cast<const Real*>(L->wrho);
  const dim3 grid = point_grid(L, 128);
  const bool res = L->grid.bc_x == RPK_BC_RESERVOIR;
  const int wm = wall_mask(L);
  if (L->streamed) {
    k_moments<Store, Real, false, 0><<<grid, 128, 0, L->stream>>>(K, pin, e, gh, rho, u, T, R, E, wcol);
  } else if (wm) {
    rpk_status st = wall_launch<Store, Real>(L, K);
    if (st != RPK_OK) return st;
    if (wm == kWallY)
      k_moments<Store, Real, true, kWallY><<<grid, 128, 0, L->stream>>>(K, pin, e, gh, rho, u, T, R, E, wcol);
    else if (wm == kWallX)
      k_moments<Store, Real, true, kWallX><<<grid, 128, 0, L->stream>>>(K, pin, e, gh, rho, u, T, R, E, wcol);
    else
      k_moments<Store, Real, true, kWallY | kWallX><<<grid, 128, 0, L->stream>>>(K, pin, e, gh, rho, u, T, R,
                                                                                E, wcol);
  } else if (res) {
    k_moments<Store, Real, true, 1><<<grid, 128, 0, L->stream>>>(K, pin, e, gh, rho, u, T, R, E, wcol);
  } else {
    k_moments<Store, Real, true, 0><<<grid, 128, 0, L->stream>>>(K, pin, e, gh, rho, u, T, R, E, wcol);
  }
  return check_launch("k_moments");
}

template <typename Store, typename Real>
rpk_status Ops<Store, Real>::diag(rpk_lattice* L, double out[8]) {
  const StepConst<Real> K = make_const<Real>(L);
  const Store* pin = static_cast<const Store*>(L->pop[L->cur]);
  const Real* e = static_cast<const Real*>(L->e);
  const Real* gh = static_cast<const Real*>(L->ghost);
  // one wave of resident blocks (4 per SM in FP32 arithmetic), grid-stride
  const int64_t need = (L->npts + kDiagThreads - 1) / kDiagThreads;
  const int64_t wave = (int64_t)L->sms * (sizeof(Real) == 4 ? 4 : 1);
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(kDiagBlocks, wave), need));
  const Real* wcol = static_cast<const Real*>(L->wrho);
  const bool res = L->grid.bc_x == RPK_BC_RESERVOIR;
  const int wm = wall_mask(L);
  bool pair = false;
  if constexpr (sizeof(Real) == 4) pair = !L->streamed && !wm && !res && L->grid.nx % 2 == 0;
  if (pair) {
    if constexpr (sizeof(Real) == 4) {
      // two points per thread (3 blocks per SM)
      const int64_t pneed = (L->npts / 2 + kDiagThreads - 1) / kDiagThreads;
      const int pblk = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(kDiagBlocks, (int64_t)L->sms * 3), pneed));
      if (L->rot_mode)
        k_diag_pair<Store, true><<<pblk, kDiagThreads, 0, L->stream>>>(K, pin, e, L->diag_partial);
      else
        k_diag_pair<Store, false><<<pblk, kDiagThreads, 0, L->stream>>>(K, pin, e, L->diag_partial);
      rpk_status st0 = check_launch("k_diag_pair");
      if (st0 != RPK_OK) return st0;
      k_diag_final<<<1, 1024, 0, L->stream>>>(L->diag_partial, pblk, L->diag_out);
      st0 = check_launch("k_diag_final");
      if (st0 != RPK_OK) return st0;
      RPK_CUDA(cudaMemcpyAsync(out, L->diag_out, kDiagVals * sizeof(double), cudaMemcpyDeviceToHost,
                               L->stream));
      RPK_CUDA(cudaStreamSynchronize(L->stream));
      return RPK_OK;
    }
  }
  if (L->streamed) {
    k_diag<Store, Real, false, 0><<<nblk, kDiagThreads, 0, L->stream>>>(K, pin, e, gh, L->diag_partial, wcol);
  } else if (wm) {
    rpk_status sw = wall_launch<Store, Real>(L, K);
    if (sw != RPK_OK) return sw;
    if (wm == kWallY)
      k_diag<Store, Real, true, kWallY><<<nblk, kDiagThreads, 0, L->stream>>>(K, pin, e, gh, L->diag_partial,
                                                                               wcol);
    else if (wm == kWallX)
      k_diag<Store, Real, true, kWallX><<<nblk, kDiagThreads, 0, L->stream>>>(K, pin, e, gh, L->diag_partial,
                                                                               wcol);
    else
      k_diag<Store, Real, true, kWallY | kWallX><<<nblk, kDiagThreads, 0, L->stream>>>(
          K, pin, e, gh, L->diag_partial, wcol);
  } else if (res) {
    k_diag<Store, Real, true, 1><<<nblk, kDiagThreads, 0, L->stream>>>(K, pin, e, gh, L->diag_partial, wcol);
  } else {
    k_diag<Store, Real, true, 0><<<nblk, kDiagThreads, 0, L->stream>>>(K, pin, e, gh, L->diag_partial, wcol);
  }
  rpk_status st = check_launch("k_diag");
  if (st != RPK_OK) return st;
  k_diag_final<<<1, 1024, 0, L->stream>>>(L->diag_partial, nblk, L->diag_out);
  st = check_launch("k_diag_final");
  if (st != RPK_OK) return st;
  RPK_CUDA(cudaMemcpyAsync(out, L->diag_out, kDiagVals * sizeof(double), cudaMemcpyDeviceToHost,
                           L->stream));
  RPK_CUDA(cudaStreamSynchronize(L->stream));
  return RPK_OK;
}

}  // namespace rpk
