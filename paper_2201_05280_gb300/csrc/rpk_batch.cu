// Batched quasi-1-D tubes: many independent nx x 1 x 1 lattices (shock tubes
// with x reservoirs) advanced by one persistent kernel launch.
//
// Each CTA takes whole tubes from a work queue (an atomic counter over a
// longest-work-first order) and runs every step of a tube itself: the pull +
// collide pass over the tube's 2 nx points reads and writes the tube's
// populations in device memory, while the auxiliary rotational energy, the
// two velocity slots, rho - 1, kappa_R, the predictor and theta_R of the tube
// live in shared memory for the whole time loop, so the transport (MacCormack
// and the FTCS sub-steps) costs no device-memory traffic. Tubes need no
// synchronisation with each other, so the launch has no grid-wide barrier. The
// arithmetic is that of the lattice kernels (k_collide, k_mac_pred,
// k_mac_corr, k_ftcs_first, k_ftcs) on an nx x 1 x 1 grid, where every y and z
// neighbour is the point itself and contributes exact zeros.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "rpk_internal.h"
#include "rpk_ops.cuh"

namespace rpk {

constexpr int kBatchArrays = 7;  // e, e*/theta, u slot 0, u slot 1, rho - 1, kappa, predictor
constexpr size_t kBatchSmemLimit = 227 * 1024;

template <typename Real>
struct TubeDev {
  StepConst<Real> K;  // nx, ny = nz = 1, n3 = nx and the relaxation constants
  Real hdt;           // dt / (2 tau1), for the initial state
  int nx, nsteps, nsub, cur;
  int streamed, pad0, pad1, pad2;
  int64_t pop_off;   // element offset of the tube in each population buffer
  int64_t pt_off;    // point offset in the concatenated point arrays
  int64_t snap_off;  // float offset of the tube's snapshots
  Real ghost[2 * kGhostStride];
};

// Gathered point index of point p (0 <= p < 2 nx) of a tube.
__device__ __forceinline__ PointIdx tube_point(int nx, int p) {
  PointIdx P;
  P.s = p >= nx;
  P.x = p - P.s * nx;
  P.y = 0;
  P.z = 0;
  P.cell = P.x;
  return P;
}

template <typename Store, typename Real, int kThreads>
__global__ void __launch_bounds__(kThreads)
    k_batch(TubeDev<Real>* __restrict__ tubes, const int* __restrict__ order, int ntubes,
            int* __restrict__ counter, Store* __restrict__ pop0, Store* __restrict__ pop1,
            Real* __restrict__ e_state, Real* __restrict__ ux_state, float* __restrict__ snaps,
            int save_every, int max_np, int implicit, unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sE = reinterpret_cast<Real*>(smem_raw);  // auxiliary E_R (state), then corrector
  Real* sS = sE + max_np;                        // e* after exchange, then theta_R
  Real* sU0 = sS + max_np;                       // u_x ring slot 0
  Real* sU1 = sU0 + max_np;                      // u_x ring slot 1
  Real* sD = sU1 + max_np;                       // rho - 1
  Real* sK = sD + max_np;                        // kappa_R
  Real* sP = sK + max_np;                        // predictor
  __shared__ int s_slot;
  const int tid = threadIdx.x;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_slot = atomicAdd(counter, 1);
    __syncthreads();
    const int slot = s_slot;
    if (slot >= ntubes) break;
    TubeDev<Real>* T = tubes + order[slot];
    const StepConst<Real> K = T->K;
    const int nx = T->nx, np = 2 * nx, nsteps = T->nsteps, nsub = T->nsub;
    const Real* ghost = T->ghost;
    const Real* gl = ghost;
    const Real* gh = ghost + kGhostStride;
    Real* gE = e_state + T->pt_off;
    Real* gU = ux_state + T->pt_off;
    for (int p = tid; p < np; p += kThreads) {
      sE[p] = gE[p];
      sU1[p] = gU[p];  // u(t-1) for the first step
    }
    int cur = T->cur;
    bool streamed = T->streamed != 0;
    Store* bufs[2] = {pop0 + T->pop_off, pop1 + T->pop_off};
    const Real t0d = K.delta * K.theta0;
    // theta_R of the two reservoirs (constant)
    const Real thGl = (Real(2) * gl[kGhE] - t0d * gl[kGhDrho]) / (K.delta * (Real(1) + gl[kGhDrho]));
    const Real thGh = (Real(2) * gh[kGhE] - t0d * gh[kGhDrho]) / (K.delta * (Real(1) + gh[kGhDrho]));
    __syncthreads();
    for (int t = 0; t < nsteps; ++t) {
      Real* uc = (t & 1) ? sU1 : sU0;
      const Real* up = (t & 1) ? sU0 : sU1;
      const Store* pin = bufs[cur];
      Store* pout = bufs[cur ^ 1];
      const bool snap = (t % save_every) == 0;
      float* sn = snaps + T->snap_off + (int64_t)(t / save_every) * 4 * np;
      // 1. pull + collide + exchange of every point of the tube
      for (int p = tid; p < np; p += kThreads) {
        const PointIdx P = tube_point(nx, p);
        Real h[kQ];
        if (streamed)
          gather<Store, Real, false, 1>(pin, ghost, K, P, h);
        else
          gather<Store, Real, true, 1>(pin, ghost, K, P, h);
        Mom<Real> m;
        const Real es = collide_point<Store, Real>(K, h, sE[p], pout + (int64_t)(P.s * kQ) * K.n3 + P.cell, m);
        sS[p] = es;
        sD[p] = m.drho;
        uc[p] = m.j[0] * m.inv_rho;
        sK[p] = K.kapc * m.rho * (K.theta0 + m.dth);
        flag_moments(m, K.theta0, status);
        if (snap) {
          sn[p] = (float)(Real(1) + m.drho);
          sn[np + p] = (float)(m.j[0] * m.inv_rho);
          sn[2 * np + p] = (float)(K.theta0 + m.dT);
          sn[3 * np + p] = (float)(Real(0.5) * K.delta * m.rho * (K.theta0 + m.dR));
        }
      }
      __syncthreads();
      // 2. MacCormack predictor (forward difference along x, same sublattice)
      for (int p = tid; p < np; p += kThreads) {
        const int s = p >= nx, x = p - s * nx;
        const Real vp = Real(1.5) * uc[p] - Real(0.5) * up[p];
        Real eq, vq;
        if (x + 1 >= nx) {
          eq = gh[kGhE];
          vq = gh[kGhU];
        } else {
          eq = sS[p + 1];
          vq = Real(1.5) * uc[p + 1] - Real(0.5) * up[p + 1];
        }
        const Real e0 = sS[p];
        Real div = Real(0);
        div += K.E0 * (vq - vp) + (eq * vq - e0 * vp);
        sP[p] = e0 - K.dt * div;
      }
      __syncthreads();
      // 3. corrector (backward difference), then theta_R of the result
      for (int p = tid; p < np; p += kThreads) {
        const int s = p >= nx, x = p - s * nx;
        const Real vp = Real(1.5) * uc[p] - Real(0.5) * up[p];
        Real eq, vq;
        if (x == 0) {
          eq = gl[kGhE];
          vq = gl[kGhU];
        } else {
          eq = sP[p - 1];
          vq = Real(1.5) * uc[p - 1] - Real(0.5) * up[p - 1];
        }
        const Real epp = sP[p];
        Real div = Real(0);
        div += K.E0 * (vp - vq) + (epp * vp - eq * vq);
        const Real val = Real(0.5) * (sS[p] + epp - K.dt * div);
        const Real dr = sD[p];
        sE[p] = val;
        sS[p] = (Real(2) * val - t0d * dr) / (K.delta * (Real(1) + dr));
      }
      __syncthreads();
      if (implicit) {
        // 4'. backward-Euler variant: per sublattice line solve
        //     (delta rho / 2) phi - dt [K+ (phi_+ - phi) - K- (phi - phi_-)] = e - delta theta0 D / 2
        //     for phi = theta_R - theta0 by cyclic reduction in shared memory:
        //     a -> sP, b -> sK, c -> sS, right-hand side and then phi -> sE.
        for (int p = tid; p < np; p += kThreads) {
          const int s = p >= nx, x = p - s * nx;
          const Real kp = sK[p];
          const Real km = x == 0 ? gl[kGhKap] : sK[p - 1];
          const Real kq = x + 1 >= nx ? gh[kGhKap] : sK[p + 1];
          sP[p] = -K.dt * Real(0.5) * (kp + km);
          sS[p] = -K.dt * Real(0.5) * (kp + kq);
        }
        __syncthreads();
        for (int p = tid; p < np; p += kThreads) {
          const int s = p >= nx, x = p - s * nx;
          const Real a = sP[p], c = sS[p], dr = sD[p];
          sK[p] = Real(0.5) * K.delta * (Real(1) + dr) - a - c;
          Real r = sE[p] - Real(0.5) * t0d * dr;
          if (x == 0) {
            r -= a * thGl;
            sP[p] = Real(0);
          }
          if (x + 1 >= nx) {
            r -= c * thGh;
            sS[p] = Real(0);
          }
          sE[p] = r;
        }
        __syncthreads();
        int h = 1;
        for (; 2 * h <= nx; h *= 2) {
          const int cnt = nx / (2 * h);  // x = 2h - 1, 4h - 1, ... < nx per line
          for (int j = tid; j < 2 * cnt; j += kThreads) {
            const int s = j >= cnt, k = j - s * cnt;
            const int x = (k + 1) * 2 * h - 1, p = s * nx + x;
            const int L = p - h;
            const Real al = -sP[p] / sK[L];
            Real a = al * sP[L], b = sK[p] + al * sS[L], c = Real(0), r = sE[p] + al * sE[L];
            if (x + h < nx) {
              const int R = p + h;
              const Real ga = -sS[p] / sK[R];
              c = ga * sS[R];
              b += ga * sP[R];
              r += ga * sE[R];
            }
            sP[p] = a;
            sK[p] = b;
            sS[p] = c;
            sE[p] = r;
          }
          __syncthreads();
        }
        // the top equation of each line, x = h - 1, is now uncoupled
        if (tid < 2) {
          const int p = tid * nx + h - 1;
          sE[p] = sE[p] / sK[p];
        }
        __syncthreads();
        for (h /= 2; h >= 1; h /= 2) {
          const int cnt = (nx + h) / (2 * h);  // x = h - 1, 3h - 1, ... < nx per line
          for (int j = tid; j < 2 * cnt; j += kThreads) {
            const int s = j >= cnt, k = j - s * cnt;
            const int x = (2 * k + 1) * h - 1, p = s * nx + x;
            Real r = sE[p];
            if (x - h >= 0) r -= sP[p] * sE[p - h];
            if (x + h < nx) r -= sS[p] * sE[p + h];
            sE[p] = r / sK[p];
          }
          __syncthreads();
        }
        for (int p = tid; p < np; p += kThreads) {
          const Real dr = sD[p];
          sE[p] = Real(0.5) * K.delta * ((Real(1) + dr) * sE[p] + K.theta0 * dr);
        }
        __syncthreads();
      } else {
        // 4. FTCS sub-steps: e += h sum_faces K_face (theta_nb - theta). The first
        //    uses theta_R of the corrector (sS) and updates e in place; later ones
        //    use theta_R = a e + c with a = 2/(delta(1 + D)), c = -delta theta0 D/(delta(1 + D))
        //    (affine in e at fixed rho), ping-ponging e between sE and sS with one
        //    barrier per sub-step.
        for (int p = tid; p < np; p += kThreads) {
          const int s = p >= nx, x = p - s * nx;
          const Real thp = sS[p], kp = sK[p];
          const Real thm = x == 0 ? thGl : sS[p - 1], km = x == 0 ? gl[kGhKap] : sK[p - 1];
          const Real thq = x + 1 >= nx ? thGh : sS[p + 1], kq = x + 1 >= nx ? gh[kGhKap] : sK[p + 1];
          Real acc = Real(0);
          acc += Real(0.5) * (kp + km) * (thm - thp);
          acc += Real(0.5) * (kp + kq) * (thq - thp);
          sE[p] = sE[p] + K.hsub * acc;
        }
        __syncthreads();
        if (nsub > 1) {
          for (int p = tid; p < np; p += kThreads) {
            const Real dr = sD[p];
            const Real inv = Real(1) / (K.delta * (Real(1) + dr));
            sP[p] = Real(2) * inv;    // a
            sD[p] = -t0d * dr * inv;  // c
          }
          __syncthreads();
          Real* ein = sE;
          Real* eout = sS;
          for (int k = 1; k < nsub; ++k) {
            for (int p = tid; p < np; p += kThreads) {
              const int s = p >= nx, x = p - s * nx;
              const Real ep = ein[p];
              const Real thp = sP[p] * ep + sD[p], kp = sK[p];
              const Real thm = x == 0 ? thGl : sP[p - 1] * ein[p - 1] + sD[p - 1];
              const Real km = x == 0 ? gl[kGhKap] : sK[p - 1];
              const Real thq = x + 1 >= nx ? thGh : sP[p + 1] * ein[p + 1] + sD[p + 1];
              const Real kq = x + 1 >= nx ? gh[kGhKap] : sK[p + 1];
              Real acc = Real(0);
              acc += Real(0.5) * (kp + km) * (thm - thp);
              acc += Real(0.5) * (kp + kq) * (thq - thp);
              eout[p] = ep + K.hsub * acc;
            }
            __syncthreads();
            Real* tmp = ein;
            ein = eout;
            eout = tmp;
          }
          if (ein != sE) {
            for (int p = tid; p < np; p += kThreads) sE[p] = ein[p];
            __syncthreads();
          }
        }
      }
      cur ^= 1;
      streamed = false;
    }
    // write the tube's state back
    const Real* ulast = (nsteps == 0) ? sU1 : (((nsteps - 1) & 1) ? sU1 : sU0);
    for (int p = tid; p < np; p += kThreads) {
      gE[p] = sE[p];
      gU[p] = ulast[p];
    }
    if (tid == 0) {
      T->cur = cur;
      T->streamed = streamed ? 1 : 0;
    }
  }
}

// Initial state and reservoir tables: one block per tube.
template <typename Store, typename Real>
__global__ void k_batch_init(TubeDev<Real>* __restrict__ tubes, const double* __restrict__ rho,
                             const double* __restrict__ u, const double* __restrict__ T,
                             const double* __restrict__ R, int64_t total_pts,
                             const double* __restrict__ res, Store* __restrict__ pop0,
                             Real* __restrict__ e_state, Real* __restrict__ ux_state) {
  TubeDev<Real>* tb = tubes + blockIdx.x;
  const StepConst<Real> K = tb->K;
  const Real hdt = tb->hdt;
  const int nx = tb->nx, np = 2 * nx;
  const int64_t off = tb->pt_off;
  Store* base = pop0 + tb->pop_off;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const PointIdx P = tube_point(nx, p);
    const int64_t g = off + p;
    Real h[kQ], e;
    init_point(K, hdt, rho[g], u[g], u[total_pts + g], u[2 * total_pts + g], T[g], R[g], h, e);
    Store* out = base + (int64_t)(P.s * kQ) * K.n3 + P.cell;
#pragma unroll
    for (int q = 0; q < kQ; ++q) out[(int64_t)q * K.n3] = from_real<Store, Real>(h[q]);
    e_state[g] = e;
    ux_state[g] = Real(u[g]);
  }
  if (threadIdx.x < 2) {
    const int side = threadIdx.x;
    const double* st = res + 12 * (int64_t)blockIdx.x + 6 * side;
    Real h[kQ], e;
    init_point(K, hdt, st[0], st[1], st[2], st[3], st[4], st[5], h, e);
    Real* gg = tb->ghost + side * kGhostStride;
    for (int q = 0; q < kQ; ++q) gg[q] = h[q];
    gg[kGhE] = e;
    gg[kGhDrho] = Real(st[0] - 1.0);
    gg[kGhU] = Real(st[1]);
    gg[kGhU + 1] = Real(st[2]);
    gg[kGhU + 2] = Real(st[3]);
    const double theta = (3.0 * st[4] + (double)K.delta * st[5]) / (3.0 + (double)K.delta);
    gg[kGhKap] = Real((double)K.kapc * st[0] * theta);
  }
  if (threadIdx.x == 0) {
    tb->cur = 0;
    tb->streamed = 1;
  }
}

// Moments of the current state, one block per tube (FP64 outputs).
template <typename Store, typename Real>
__global__ void k_batch_moments(const TubeDev<Real>* __restrict__ tubes, const Store* __restrict__ pop0,
                                const Store* __restrict__ pop1, const Real* __restrict__ e_state,
                                int64_t total_pts, double* __restrict__ out) {
  const TubeDev<Real>* tb = tubes + blockIdx.x;
  const StepConst<Real> K = tb->K;
  const int nx = tb->nx, np = 2 * nx;
  const Store* pin = (tb->cur ? pop1 : pop0) + tb->pop_off;
  const int64_t off = tb->pt_off;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const PointIdx P = tube_point(nx, p);
    Real h[kQ];
    if (tb->streamed)
      gather<Store, Real, false, 1>(pin, tb->ghost, K, P, h);
    else
      gather<Store, Real, true, 1>(pin, tb->ghost, K, P, h);
    Mom<Real> m;
    raw_moments(h, m);
    recover(m, e_state[off + p], K);
    const int64_t g = off + p;
    out[g] = 1.0 + (double)m.drho;
    out[total_pts + g] = (double)(m.j[0] * m.inv_rho);
    out[2 * total_pts + g] = (double)(m.j[1] * m.inv_rho);
    out[3 * total_pts + g] = (double)(m.j[2] * m.inv_rho);
    out[4 * total_pts + g] = (double)K.theta0 + (double)m.dT;
    out[5 * total_pts + g] = (double)K.theta0 + (double)m.dR;
    out[6 * total_pts + g] =
        0.5 * (double)K.delta * (1.0 + (double)m.drho) * ((double)K.theta0 + (double)m.dR);
  }
}

// Moment blocks (per tube [4][2 nx] floats: rho, u_x, theta_T, E_R, at float
// offset 4 pt_off) -> the FP64 staging rows read by k_batch_init (rho, u (3
// rows), theta_T, theta_R). theta_R = 2 E_R / (delta rho); theta_T when delta = 0.
// Non-positive or non-finite values set bit 2 of the status word.
template <typename Real>
__global__ void k_state_to_stage(const TubeDev<Real>* __restrict__ tubes, const float* __restrict__ state,
                                 int64_t n, double* __restrict__ stage, unsigned* __restrict__ status) {
  const TubeDev<Real>* tb = tubes + blockIdx.x;
  const int np = 2 * tb->nx;
  const int64_t off = tb->pt_off;
  const float* s = state + 4 * off;
  const double delta = (double)tb->K.delta;
  bool bad = false;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const double rho = s[p], ux = s[np + p], T = s[2 * np + p], er = s[3 * np + p];
    const double R = delta > 0.0 ? 2.0 * er / (delta * rho) : T;
    bad |= !(rho > 0.0) || !(T > 0.0) || !(R > 0.0) || !isfinite(rho) || !isfinite(ux) ||
           !isfinite(T) || !isfinite(R);
    stage[off + p] = rho;
    stage[n + off + p] = ux;
    stage[2 * n + off + p] = 0.0;
    stage[3 * n + off + p] = 0.0;
    stage[4 * n + off + p] = T;
    stage[5 * n + off + p] = R;
  }
  if (bad) atomicOr(status, 4u);
}

// FP64 moment rows of k_batch_moments -> moment blocks (rho, u_x, theta_T, E_R).
template <typename Real>
__global__ void k_stage_to_state(const TubeDev<Real>* __restrict__ tubes, const double* __restrict__ stage,
                                 int64_t n, float* __restrict__ state) {
  const TubeDev<Real>* tb = tubes + blockIdx.x;
  const int np = 2 * tb->nx;
  const int64_t off = tb->pt_off;
  float* s = state + 4 * off;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    s[p] = (float)stage[off + p];
    s[np + p] = (float)stage[n + off + p];
    s[2 * np + p] = (float)stage[4 * n + off + p];
    s[3 * np + p] = (float)stage[6 * n + off + p];
  }
}

template <typename Real>
__global__ void k_set_steps(TubeDev<Real>* __restrict__ tubes, const int* __restrict__ nsteps, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) tubes[i].nsteps = nsteps[i];
}

}  // namespace rpk

using namespace rpk;

struct rpk_batch {
  int precision = RPK_F32, ntubes = 0, save_every = 1, device = 0;
  cudaStream_t stream = nullptr;
  std::vector<rpk_tube> tubes;
  std::vector<int> nsub;
  std::vector<int64_t> pt_off, snap_off;
  int64_t total_pts = 0, pop_elems = 0, snap_floats = 0;
  int max_nx = 0;
  size_t real_elem = 4, store_elem = 4;
  void* pop[2] = {nullptr, nullptr};
  void* e_state = nullptr;
  void* ux_state = nullptr;
  void* tubes_dev = nullptr;
  int* order_dev = nullptr;
  int* counter = nullptr;
  float* snaps = nullptr;
  unsigned* status = nullptr;
  double* stage = nullptr;  // 7 x total_pts doubles, for init and reads
  double* res_dev = nullptr;  // 12 reservoir values per tube
  int* steps_dev = nullptr;   // per-tube step counts for rpk_batch_set_steps
  std::vector<int> max_steps; // step counts given at creation (bound the snapshot storage)
  bool nsub_ok = false;       // every tube's FTCS sub-step count is resolved
  int implicit = 0;           // rotational diffusion: 0 FTCS sub-steps, 1 backward Euler
  bool init_ok = false;
  int threads = 256, ctas_per_sm = 1;
  cudaGraphExec_t graph = nullptr;
  int graph_threads = 0, graph_ctas = 0, graph_implicit = 0;
};

namespace {

template <typename Store, typename Real>
struct BatchOps {
  static void* kernel(int threads) {
    switch (threads) {
      case 128: return (void*)k_batch<Store, Real, 128>;
      case 256: return (void*)k_batch<Store, Real, 256>;
      case 384: return (void*)k_batch<Store, Real, 384>;
      case 512: return (void*)k_batch<Store, Real, 512>;
      default: return nullptr;
    }
  }
};

bool supported_threads(int t) { return t == 128 || t == 256 || t == 384 || t == 512; }

size_t batch_smem(const rpk_batch* B) {
  return (size_t)kBatchArrays * 2 * B->max_nx * B->real_elem;
}

template <typename F>
rpk_status with_batch_types(int precision, F&& f) {
  if (precision == RPK_F64) return f(BatchOps<double, double>{}, (double*)nullptr);
  return f(BatchOps<float, float>{}, (float*)nullptr);
}

void free_batch(rpk_batch* B) {
  if (B->graph) cudaGraphExecDestroy(B->graph);
  void* ptrs[] = {B->pop[0], B->pop[1], B->e_state, B->ux_state, B->tubes_dev, B->order_dev,
                  B->counter, B->snaps,  B->status, B->stage,    B->res_dev,   B->steps_dev};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

rpk_status dev_alloc(void** p, size_t bytes) {
  cudaError_t err = cudaMalloc(p, bytes);
  if (err != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(err == cudaErrorMemoryAllocation ? RPK_ERR_OOM : RPK_ERR_CUDA,
                std::string("batch allocation failed: ") + cudaGetErrorString(err));
  }
  return RPK_OK;
}

// Work order of the queue: longest work first (collide work ~ points x steps,
// diffusion ~ points x steps x nsub).
rpk_status upload_order(rpk_batch* B) {
  std::vector<int> order(B->ntubes);
  for (int i = 0; i < B->ntubes; ++i) order[i] = i;
  std::vector<double> work(B->ntubes);
  for (int i = 0; i < B->ntubes; ++i)
    work[i] = 2.0 * B->tubes[i].nx * B->tubes[i].nsteps * (8.0 + (B->implicit ? 4.0 : B->nsub[i]));
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
  RPK_CUDA(cudaMemcpyAsync(B->order_dev, order.data(), sizeof(int) * B->ntubes,
                           cudaMemcpyHostToDevice, B->stream));
  RPK_CUDA(cudaStreamSynchronize(B->stream));
  return RPK_OK;
}

// Upload the tube descriptors (constants, offsets, nsub) and the work order.
template <typename Real>
rpk_status upload_tubes(rpk_batch* B) {
  std::vector<TubeDev<Real>> td(B->ntubes);
  int64_t pop_off = 0;
  for (int i = 0; i < B->ntubes; ++i) {
    const rpk_tube& t = B->tubes[i];
    TubeDev<Real>& d = td[i];
    std::memset(&d, 0, sizeof(d));
    d.K = make_step_const<Real>(t.relax, B->nsub[i], t.nx, 1, 1);
    d.hdt = Real(0.5 * t.relax.dt / t.relax.tau1);
    d.nx = t.nx;
    d.nsteps = t.nsteps;
    d.nsub = B->nsub[i];
    d.cur = 0;
    d.streamed = 1;
    d.pop_off = pop_off;
    d.pt_off = B->pt_off[i];
    d.snap_off = B->snap_off[i];
    pop_off += (int64_t)2 * kQ * t.nx;
  }
  RPK_CUDA(cudaMemcpyAsync(B->tubes_dev, td.data(), sizeof(TubeDev<Real>) * B->ntubes,
                           cudaMemcpyHostToDevice, B->stream));
  RPK_CUDA(cudaStreamSynchronize(B->stream));
  return upload_order(B);
}

// Shared-memory limit of the kernel variant (outside any stream capture).
template <typename Store, typename Real>
rpk_status prepare_batch(rpk_batch* B, int threads) {
  void* kfn = BatchOps<Store, Real>::kernel(threads);
  if (!kfn) return fail(RPK_ERR_ARG, "unsupported thread count");
  RPK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)batch_smem(B)));
  return RPK_OK;
}

template <typename Store, typename Real>
rpk_status launch_batch(rpk_batch* B, cudaStream_t stream, int threads, int ctas_per_sm) {
  int nsm = 0;
  RPK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, B->device));
  const size_t smem = batch_smem(B);
  const int grid = std::max(1, std::min(B->ntubes, nsm * ctas_per_sm));
  RPK_CUDA(cudaMemsetAsync(B->counter, 0, sizeof(int), stream));
  TubeDev<Real>* tubes = static_cast<TubeDev<Real>*>(B->tubes_dev);
  Store* p0 = static_cast<Store*>(B->pop[0]);
  Store* p1 = static_cast<Store*>(B->pop[1]);
  Real* es = static_cast<Real*>(B->e_state);
  Real* us = static_cast<Real*>(B->ux_state);
  const int max_np = 2 * B->max_nx;
  switch (threads) {
#define RPK_LAUNCH(NT)                                                                         \
  case NT:                                                                                     \
    k_batch<Store, Real, NT><<<grid, NT, smem, stream>>>(tubes, B->order_dev, B->ntubes,       \
                                                         B->counter, p0, p1, es, us, B->snaps, \
                                                         B->save_every, max_np, B->implicit,   \
                                                         B->status);                           \
    break;
    RPK_LAUNCH(128)
    RPK_LAUNCH(256)
    RPK_LAUNCH(384)
    RPK_LAUNCH(512)
#undef RPK_LAUNCH
  }
  RPK_CUDA(cudaGetLastError());
  return RPK_OK;
}

// Tube descriptors, then the initial state from the staging rows (filled from
// host fields before the call, or from device moment blocks here).
rpk_status init_from_stage(rpk_batch* B, const float* state) {
  const int64_t n = B->total_pts;
  double* s = B->stage;
  rpk_status st = with_batch_types(B->precision, [&](auto ops, auto* real_tag) {
    using Real = std::remove_pointer_t<decltype(real_tag)>;
    return upload_tubes<Real>(B);
  });
  if (st != RPK_OK) return st;
  RPK_CUDA(cudaMemsetAsync(B->status, 0, sizeof(unsigned), B->stream));
  if (B->precision == RPK_F64) {
    auto* td = static_cast<TubeDev<double>*>(B->tubes_dev);
    if (state) k_state_to_stage<double><<<B->ntubes, 256, 0, B->stream>>>(td, state, n, s, B->status);
    k_batch_init<double, double><<<B->ntubes, 256, 0, B->stream>>>(
        td, s, s + n, s + 4 * n, s + 5 * n, n, B->res_dev, static_cast<double*>(B->pop[0]),
        static_cast<double*>(B->e_state), static_cast<double*>(B->ux_state));
  } else {
    auto* td = static_cast<TubeDev<float>*>(B->tubes_dev);
    if (state) k_state_to_stage<float><<<B->ntubes, 256, 0, B->stream>>>(td, state, n, s, B->status);
    k_batch_init<float, float><<<B->ntubes, 256, 0, B->stream>>>(
        td, s, s + n, s + 4 * n, s + 5 * n, n, B->res_dev, static_cast<float*>(B->pop[0]),
        static_cast<float*>(B->e_state), static_cast<float*>(B->ux_state));
  }
  RPK_CUDA(cudaGetLastError());
  RPK_CUDA(cudaStreamSynchronize(B->stream));
  B->init_ok = true;
  return RPK_OK;
}

bool config_fits(const rpk_batch* B, int threads, int ctas) {
  return supported_threads(threads) && ctas >= 1 && batch_smem(B) * ctas <= kBatchSmemLimit &&
         threads * ctas <= 2048;
}

}  // namespace

extern "C" {

int rpk_batch_max_nx(int precision) {
  const size_t real = precision == RPK_F64 ? 8 : 4;
  return (int)((kBatchSmemLimit - 1024) / (kBatchArrays * 2 * real));
}

rpk_status rpk_batch_create(int precision, int ntubes, const rpk_tube* tubes, int save_every,
                            void* cuda_stream, rpk_batch** out) {
  if (!out || !tubes) return fail(RPK_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (precision != RPK_F64 && precision != RPK_F32)
    return fail(RPK_ERR_ARG, "batched tubes support RPK_F64 and RPK_F32");
  if (ntubes < 1) return fail(RPK_ERR_ARG, "ntubes must be >= 1");
  if (save_every < 1) return fail(RPK_ERR_ARG, "save_every must be >= 1");
  const int max_nx = rpk_batch_max_nx(precision);
  for (int i = 0; i < ntubes; ++i) {
    const rpk_tube& t = tubes[i];
    if (t.nx < 2 || t.nx > max_nx)
      return fail(RPK_ERR_ARG, "tube " + std::to_string(i) + ": nx must lie in [2, " +
                                   std::to_string(max_nx) + "] for this precision");
    if (t.nsteps < 0) return fail(RPK_ERR_ARG, "tube " + std::to_string(i) + ": nsteps < 0");
    rpk_status st = validate_relax(&t.relax);
    if (st != RPK_OK) return fail(st, "tube " + std::to_string(i) + ": " + rpk_last_error());
    for (int side = 0; side < 2; ++side) {
      const double* r = t.res + 6 * side;
      if (!(r[0] > 0.0) || !(r[4] > 0.0) || !(r[5] > 0.0))
        return fail(RPK_ERR_PARAM, "tube " + std::to_string(i) + ": reservoir rho, theta must be > 0");
    }
  }
  rpk_batch* B = new (std::nothrow) rpk_batch();
  if (!B) return fail(RPK_ERR_OOM, "host allocation failed");
  B->precision = precision;
  B->ntubes = ntubes;
  B->save_every = save_every;
  B->stream = static_cast<cudaStream_t>(cuda_stream);
  B->tubes.assign(tubes, tubes + ntubes);
  B->nsub.assign(ntubes, 1);
  B->real_elem = B->store_elem = precision == RPK_F64 ? 8 : 4;
  cudaError_t err = cudaGetDevice(&B->device);
  if (err != cudaSuccess) {
    delete B;
    return cuda_fail(err, "cudaGetDevice");
  }
  B->pt_off.resize(ntubes);
  B->snap_off.resize(ntubes);
  for (int i = 0; i < ntubes; ++i) {
    B->pt_off[i] = B->total_pts;
    B->snap_off[i] = B->snap_floats;
    const int64_t np = 2 * (int64_t)tubes[i].nx;
    const int64_t nsnap = (tubes[i].nsteps + save_every - 1) / save_every;
    B->total_pts += np;
    B->snap_floats += nsnap * 4 * np;
    B->max_nx = std::max(B->max_nx, tubes[i].nx);
  }
  B->pop_elems = (int64_t)kQ * B->total_pts;
  const size_t tube_bytes = precision == RPK_F64 ? sizeof(TubeDev<double>) : sizeof(TubeDev<float>);
  rpk_status st = RPK_OK;
  if (st == RPK_OK) st = dev_alloc(&B->pop[0], B->pop_elems * B->store_elem);
  if (st == RPK_OK) st = dev_alloc(&B->pop[1], B->pop_elems * B->store_elem);
  if (st == RPK_OK) st = dev_alloc(&B->e_state, B->total_pts * B->real_elem);
  if (st == RPK_OK) st = dev_alloc(&B->ux_state, B->total_pts * B->real_elem);
  if (st == RPK_OK) st = dev_alloc(&B->tubes_dev, tube_bytes * ntubes);
  if (st == RPK_OK) st = dev_alloc((void**)&B->order_dev, sizeof(int) * ntubes);
  if (st == RPK_OK) st = dev_alloc((void**)&B->counter, sizeof(int));
  if (st == RPK_OK) st = dev_alloc((void**)&B->snaps, std::max<int64_t>(1, B->snap_floats) * sizeof(float));
  if (st == RPK_OK) st = dev_alloc((void**)&B->status, sizeof(unsigned));
  if (st == RPK_OK) st = dev_alloc((void**)&B->stage, sizeof(double) * 7 * B->total_pts);
  if (st == RPK_OK) st = dev_alloc((void**)&B->res_dev, sizeof(double) * 12 * ntubes);
  if (st == RPK_OK) st = dev_alloc((void**)&B->steps_dev, sizeof(int) * ntubes);
  if (st == RPK_OK) {
    std::vector<double> res(12 * (size_t)ntubes);
    for (int i = 0; i < ntubes; ++i) std::memcpy(&res[12 * (size_t)i], tubes[i].res, 12 * sizeof(double));
    cudaError_t e = cudaMemcpyAsync(B->res_dev, res.data(), res.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "rpk_batch_create");
  }
  if (st != RPK_OK) {
    free_batch(B);
    delete B;
    return st;
  }
  B->max_steps.resize(ntubes);
  B->nsub_ok = true;
  for (int i = 0; i < ntubes; ++i) {
    B->max_steps[i] = tubes[i].nsteps;
    if (tubes[i].relax.nsub > 0)
      B->nsub[i] = tubes[i].relax.nsub;
    else
      B->nsub_ok = false;
  }
  *out = B;
  return RPK_OK;
}

void rpk_batch_destroy(rpk_batch* B) {
  if (!B) return;
  cudaStreamSynchronize(B->stream);
  free_batch(B);
  delete B;
}

rpk_status rpk_batch_init(rpk_batch* B, const double* rho, const double* u, const double* T,
                          const double* R) {
  if (!B || !rho || !u || !T || !R) return fail(RPK_ERR_ARG, "NULL argument");
  RPK_CUDA(cudaSetDevice(B->device));
  const int64_t n = B->total_pts;
  for (int64_t p = 0; p < n; ++p)
    if (!(rho[p] > 0.0) || !(T[p] > 0.0) || !(R[p] > 0.0) || !std::isfinite(rho[p]) ||
        !std::isfinite(T[p]) || !std::isfinite(R[p]))
      return fail(RPK_ERR_PARAM, "fields need finite rho > 0, theta_T > 0, theta_R > 0");
  for (int64_t p = 0; p < 3 * n; ++p)
    if (!std::isfinite(u[p])) return fail(RPK_ERR_PARAM, "u not finite");
  // FTCS sub-steps per tube (rpk_auto_nsub with one active axis when nsub = 0)
  for (int i = 0; i < B->ntubes; ++i) {
    const rpk_tube& t = B->tubes[i];
    if (t.relax.nsub > 0) {
      B->nsub[i] = t.relax.nsub;
      continue;
    }
    double tmax = 0.0;
    for (int64_t p = B->pt_off[i]; p < B->pt_off[i] + 2 * t.nx; ++p)
      tmax = std::max(tmax, (3.0 * T[p] + t.relax.delta * R[p]) / (3.0 + t.relax.delta));
    for (int side = 0; side < 2; ++side)
      tmax = std::max(tmax, (3.0 * t.res[6 * side + 4] + t.relax.delta * t.res[6 * side + 5]) /
                                (3.0 + t.relax.delta));
    B->nsub[i] = rpk_auto_nsub(&t.relax, tmax, 1);
  }
  B->nsub_ok = true;
  double* s = B->stage;
  RPK_CUDA(cudaMemcpyAsync(s, rho, n * sizeof(double), cudaMemcpyHostToDevice, B->stream));
  RPK_CUDA(cudaMemcpyAsync(s + n, u, 3 * n * sizeof(double), cudaMemcpyHostToDevice, B->stream));
  RPK_CUDA(cudaMemcpyAsync(s + 4 * n, T, n * sizeof(double), cudaMemcpyHostToDevice, B->stream));
  RPK_CUDA(cudaMemcpyAsync(s + 5 * n, R, n * sizeof(double), cudaMemcpyHostToDevice, B->stream));
  return init_from_stage(B, nullptr);
}

rpk_status rpk_batch_init_device(rpk_batch* B, const float* state) {
  if (!B || !state) return fail(RPK_ERR_ARG, "NULL argument");
  if (!B->nsub_ok)
    return fail(RPK_ERR_STATE, "FTCS sub-step counts unresolved: give relax.nsub > 0 for every "
                               "tube or initialise once from host fields");
  RPK_CUDA(cudaSetDevice(B->device));
  return init_from_stage(B, state);
}

rpk_status rpk_batch_set_steps(rpk_batch* B, const int* nsteps) {
  if (!B || !nsteps) return fail(RPK_ERR_ARG, "NULL argument");
  for (int i = 0; i < B->ntubes; ++i)
    if (nsteps[i] < 0 || nsteps[i] > B->max_steps[i])
      return fail(RPK_ERR_ARG, "tube " + std::to_string(i) + ": nsteps must lie in [0, " +
                                   std::to_string(B->max_steps[i]) + "] (its count at creation)");
  RPK_CUDA(cudaSetDevice(B->device));
  for (int i = 0; i < B->ntubes; ++i) B->tubes[i].nsteps = nsteps[i];
  if (!B->init_ok) return RPK_OK;  // uploaded with the tube descriptors at initialisation
  RPK_CUDA(cudaMemcpyAsync(B->steps_dev, nsteps, sizeof(int) * B->ntubes, cudaMemcpyHostToDevice,
                           B->stream));
  const int blocks = (B->ntubes + 255) / 256;
  if (B->precision == RPK_F64)
    k_set_steps<double><<<blocks, 256, 0, B->stream>>>(static_cast<TubeDev<double>*>(B->tubes_dev),
                                                        B->steps_dev, B->ntubes);
  else
    k_set_steps<float><<<blocks, 256, 0, B->stream>>>(static_cast<TubeDev<float>*>(B->tubes_dev),
                                                       B->steps_dev, B->ntubes);
  RPK_CUDA(cudaGetLastError());
  return upload_order(B);  // synchronises the stream
}

rpk_status rpk_batch_moments_device(rpk_batch* B, float* state) {
  if (!B || !state) return fail(RPK_ERR_ARG, "NULL argument");
  if (!B->init_ok) return fail(RPK_ERR_STATE, "initialise the batch first");
  RPK_CUDA(cudaSetDevice(B->device));
  const int64_t n = B->total_pts;
  if (B->precision == RPK_F64) {
    const auto* td = static_cast<const TubeDev<double>*>(B->tubes_dev);
    k_batch_moments<double, double><<<B->ntubes, 256, 0, B->stream>>>(
        td, static_cast<const double*>(B->pop[0]), static_cast<const double*>(B->pop[1]),
        static_cast<const double*>(B->e_state), n, B->stage);
    k_stage_to_state<double><<<B->ntubes, 256, 0, B->stream>>>(td, B->stage, n, state);
  } else {
    const auto* td = static_cast<const TubeDev<float>*>(B->tubes_dev);
    k_batch_moments<float, float><<<B->ntubes, 256, 0, B->stream>>>(
        td, static_cast<const float*>(B->pop[0]), static_cast<const float*>(B->pop[1]),
        static_cast<const float*>(B->e_state), n, B->stage);
    k_stage_to_state<float><<<B->ntubes, 256, 0, B->stream>>>(td, B->stage, n, state);
  }
  RPK_CUDA(cudaGetLastError());
  return RPK_OK;
}

rpk_status rpk_batch_set_diffusion(rpk_batch* B, int mode) {
  if (!B) return fail(RPK_ERR_ARG, "NULL batch");
  if (mode != 0 && mode != 1) return fail(RPK_ERR_ARG, "mode must be 0 (FTCS) or 1 (backward Euler)");
  B->implicit = mode;
  return RPK_OK;
}

rpk_status rpk_batch_set_config(rpk_batch* B, int threads, int ctas_per_sm) {
  if (!B) return fail(RPK_ERR_ARG, "NULL batch");
  if (!config_fits(B, threads, ctas_per_sm))
    return fail(RPK_ERR_ARG, "unsupported configuration (threads in {128,256,384,512}; shared "
                             "memory of the CTAs per SM must fit)");
  B->threads = threads;
  B->ctas_per_sm = ctas_per_sm;
  return RPK_OK;
}

rpk_status rpk_batch_run(rpk_batch* B) {
  if (!B) return fail(RPK_ERR_ARG, "NULL batch");
  if (!B->init_ok) return fail(RPK_ERR_STATE, "initialise the batch first");
  RPK_CUDA(cudaSetDevice(B->device));
  if (!B->graph || B->graph_threads != B->threads || B->graph_ctas != B->ctas_per_sm ||
      B->graph_implicit != B->implicit) {
    if (B->graph) {
      cudaGraphExecDestroy(B->graph);
      B->graph = nullptr;
    }
    rpk_status pst = with_batch_types(B->precision, [&](auto ops, auto* real_tag) {
      using Real = std::remove_pointer_t<decltype(real_tag)>;
      return prepare_batch<Real, Real>(B, B->threads);
    });
    if (pst != RPK_OK) return pst;
    cudaStream_t cap = nullptr;
    RPK_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    rpk_status st = RPK_OK;
    if (err == cudaSuccess) {
      st = with_batch_types(B->precision, [&](auto ops, auto* real_tag) {
        using Real = std::remove_pointer_t<decltype(real_tag)>;
        return launch_batch<Real, Real>(B, cap, B->threads, B->ctas_per_sm);
      });
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(cap, &g);
      if (st == RPK_OK && e2 == cudaSuccess) e2 = cudaGraphInstantiate(&B->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      err = e2;
    }
    cudaStreamDestroy(cap);
    if (st != RPK_OK) return st;
    if (err != cudaSuccess) return cuda_fail(err, "batch graph capture");
    B->graph_threads = B->threads;
    B->graph_ctas = B->ctas_per_sm;
    B->graph_implicit = B->implicit;
  }
  RPK_CUDA(cudaGraphLaunch(B->graph, B->stream));
  return RPK_OK;
}

rpk_status rpk_batch_read_moments(rpk_batch* B, double* rho, double* u, double* T, double* R,
                                  double* E) {
  if (!B) return fail(RPK_ERR_ARG, "NULL batch");
  if (!B->init_ok) return fail(RPK_ERR_STATE, "initialise the batch first");
  RPK_CUDA(cudaSetDevice(B->device));
  const int64_t n = B->total_pts;
  if (B->precision == RPK_F64)
    k_batch_moments<double, double><<<B->ntubes, 256, 0, B->stream>>>(
        static_cast<const TubeDev<double>*>(B->tubes_dev), static_cast<const double*>(B->pop[0]),
        static_cast<const double*>(B->pop[1]), static_cast<const double*>(B->e_state), n, B->stage);
  else
    k_batch_moments<float, float><<<B->ntubes, 256, 0, B->stream>>>(
        static_cast<const TubeDev<float>*>(B->tubes_dev), static_cast<const float*>(B->pop[0]),
        static_cast<const float*>(B->pop[1]), static_cast<const float*>(B->e_state), n, B->stage);
  RPK_CUDA(cudaGetLastError());
  const size_t b = n * sizeof(double);
  if (rho) RPK_CUDA(cudaMemcpyAsync(rho, B->stage, b, cudaMemcpyDeviceToHost, B->stream));
  if (u) RPK_CUDA(cudaMemcpyAsync(u, B->stage + n, 3 * b, cudaMemcpyDeviceToHost, B->stream));
  if (T) RPK_CUDA(cudaMemcpyAsync(T, B->stage + 4 * n, b, cudaMemcpyDeviceToHost, B->stream));
  if (R) RPK_CUDA(cudaMemcpyAsync(R, B->stage + 5 * n, b, cudaMemcpyDeviceToHost, B->stream));
  if (E) RPK_CUDA(cudaMemcpyAsync(E, B->stage + 6 * n, b, cudaMemcpyDeviceToHost, B->stream));
  unsigned flags = 0;
  RPK_CUDA(cudaMemcpyAsync(&flags, B->status, sizeof(unsigned), cudaMemcpyDeviceToHost, B->stream));
  RPK_CUDA(cudaStreamSynchronize(B->stream));
  if (flags) return fail(RPK_ERR_NUMERIC, "a tube flagged a non-finite or non-positive moment");
  return RPK_OK;
}

rpk_status rpk_batch_snapshots(rpk_batch* B, float* out, int64_t* count) {
  if (!B || !count) return fail(RPK_ERR_ARG, "NULL argument");
  RPK_CUDA(cudaSetDevice(B->device));
  *count = B->snap_floats;
  if (out && B->snap_floats > 0) {
    RPK_CUDA(cudaMemcpyAsync(out, B->snaps, B->snap_floats * sizeof(float), cudaMemcpyDeviceToHost,
                             B->stream));
    RPK_CUDA(cudaStreamSynchronize(B->stream));
  }
  return RPK_OK;
}

rpk_status rpk_batch_autotune(rpk_batch* B, int64_t out[3]) {
  if (!B || !out) return fail(RPK_ERR_ARG, "NULL argument");
  if (!B->init_ok) return fail(RPK_ERR_STATE, "initialise the batch first");
  RPK_CUDA(cudaSetDevice(B->device));
  int nsm = 0;
  RPK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, B->device));
  // sample: up to 2 tubes per SM spread over the work order, 32 steps each, at rest
  const int nsample = std::min(B->ntubes, 2 * nsm);
  std::vector<rpk_tube> tv;
  for (int i = 0; i < nsample; ++i) {
    rpk_tube t = B->tubes[(int64_t)i * B->ntubes / nsample];
    t.nsteps = std::min(t.nsteps, 32);
    t.relax.nsub = B->nsub[(int64_t)i * B->ntubes / nsample];
    tv.push_back(t);
  }
  rpk_batch* S = nullptr;
  rpk_status st = rpk_batch_create(B->precision, nsample, tv.data(), 1 << 30, B->stream, &S);
  if (st != RPK_OK) return st;
  S->max_nx = B->max_nx;  // same shared-memory footprint as the real launch
  S->implicit = B->implicit;
  std::vector<double> rho(S->total_pts, 1.0), u(3 * S->total_pts, 0.0), T(S->total_pts, kTheta0);
  st = rpk_batch_init(S, rho.data(), u.data(), T.data(), T.data());
  double best_ms = 1e300;
  int best_t = B->threads, best_c = B->ctas_per_sm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == RPK_OK) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cand_t[] = {128, 256, 384, 512};
    for (int t : cand_t) {
      for (int c = 1; c <= 4; ++c) {
        if (!config_fits(S, t, c)) continue;
        float ms = 0.f;
        st = with_batch_types(B->precision, [&](auto ops, auto* real_tag) {
          using Real = std::remove_pointer_t<decltype(real_tag)>;
          return prepare_batch<Real, Real>(S, t);
        });
        for (int rep = 0; rep < 2 && st == RPK_OK; ++rep) {
          cudaEventRecord(e0, B->stream);
          st = with_batch_types(B->precision, [&](auto ops, auto* real_tag) {
            using Real = std::remove_pointer_t<decltype(real_tag)>;
            return launch_batch<Real, Real>(S, B->stream, t, c);
          });
          cudaEventRecord(e1, B->stream);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&ms, e0, e1);
        }
        if (st != RPK_OK) break;
        if (ms < best_ms) {
          best_ms = ms;
          best_t = t;
          best_c = c;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  rpk_batch_destroy(S);
  if (st != RPK_OK) return st;
  B->threads = best_t;
  B->ctas_per_sm = best_c;
  out[0] = best_t;
  out[1] = best_c;
  out[2] = (int64_t)(best_ms * 1000.0);
  return RPK_OK;
}

}  // extern "C"
