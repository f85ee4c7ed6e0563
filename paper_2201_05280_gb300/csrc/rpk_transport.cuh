// Fused rotational transport of one step on a periodic grid (Sec. 5, the
// advection-diffusion of the rotational energy): MacCormack predictor,
// corrector and the first FTCS sub-step of the flux-form equations in one pass
// over HBM.
//
// The three-pass form (k_mac_pred, k_mac_corr, k_ftcs_first) stores the
// predictor, the advecting velocity, the corrector and theta_R between passes
// and reads them back: 92 B per point in FP32. This kernel reads each input
// field once -- Er* (after the exchange), u(t), u(t-1), rho - 1 and kappa_R,
// 36 B -- and writes the new Er, 4 B. The intermediates live in shared memory.
//
// Each block owns a TX x TY tile of one sublattice and marches along z through
// a chunk of planes, keeping rings of planes in shared memory:
//   front  Er*, v = (3 u(t) - u(t-1))/2 of plane k+1 on the tile + 2 halo
//   pred   ep = Er* - dt div(Er* v) (forward differences) of plane k on the
//          tile + [-2, +1] halo
//   corr   Er' = (Er* + ep - dt div(ep v))/2 (backward differences) and
//          theta_R = (2 Er' - delta theta0 drho)/(delta (1 + drho)) of plane k
//          on the tile + 1 halo
//   ftcs   Er'' = Er' + hsub sum_faces (kappa_p + kappa_q)/2 (theta_q - theta_p)
//          of plane k - 1 on the tile, written to HBM
// The halos are recomputed by the neighbouring tiles (1.4x the arithmetic of
// the tile itself, served from L2 and shared memory, not HBM). Arithmetic and
// its order are those of the three-pass kernels.
#pragma once

#include "rpk_kernels.cuh"

namespace rpk {

constexpr int kFTX = 32, kFTY = 16, kFThreads = 256;
constexpr int kFP3 = kFTX + 4, kFR3 = kFP3 * (kFTY + 4);  // front: x, y in [-2, T + 2)
constexpr int kFP2 = kFTX + 3, kFR2 = kFP2 * (kFTY + 3);  // predictor: [-2, T + 1)
constexpr int kFP1 = kFTX + 2, kFR1 = kFP1 * (kFTY + 2);  // corrector, theta_R, kappa_R: [-1, T + 1)
constexpr int kFT = kFTX * kFTY;

template <typename Real>
struct FusedSmem {
  Real es[2][kFR3];         // Er* (deviation), planes k, k+1
  Real vx[2][kFR3];         // advecting velocity, planes k, k+1
  Real vy[2][kFR3];
  Real vz[3][kFR3];         // planes k-1, k, k+1
  Real ep[2][kFR2];         // predictor, planes k-1, k
  Real th[3][kFR1];         // theta_R - theta0 after the corrector, planes k-2 .. k
  Real kap[4][kFR1];        // kappa_R, planes k-2 .. k (a fourth slot is being filled)
  Real dr[kFR1];            // rho - 1 of plane k
  Real ec[2][kFT];          // corrector result on the tile, planes k-1, k
  int gx[kFP3];             // global x of local column lx (x0 - 2 + lx, wrapped)
  int gy[kFTY + 4];         // global y * nx of local row ly (y0 - 2 + ly, wrapped)
};

__device__ __forceinline__ int pmod(int a, int n) {
  const int r = a % n;
  return r < 0 ? r + n : r;
}

// blockIdx.x: tile (x fastest, then y) and sublattice; blockIdx.y: z chunk of
// zchunk output planes. e_next receives Er after the first FTCS sub-step.
template <typename Real>
__global__ void __launch_bounds__(kFThreads, sizeof(Real) == 4 ? 4 : 2)
    k_transport_fused(StepConst<Real> K, const Real* __restrict__ es_g,
                      const Real* __restrict__ ucur, const Real* __restrict__ uprev,
                      const Real* __restrict__ drho_g, const Real* __restrict__ kap_g,
                      Real* __restrict__ e_next, int zchunk) {
  extern __shared__ __align__(16) unsigned char fused_smem_raw[];
  FusedSmem<Real>& S = *reinterpret_cast<FusedSmem<Real>*>(fused_smem_raw);
  const int nx = K.nx, ny = K.ny, nz = K.nz;
  const int ntx = (nx + kFTX - 1) / kFTX, nty = (ny + kFTY - 1) / kFTY;
  int b = blockIdx.x;
  const int tx = b % ntx;
  b /= ntx;
  const int ty = b % nty;
  const int s = b / nty;
  const int x0 = tx * kFTX, y0 = ty * kFTY;
  const int z0 = blockIdx.y * zchunk;
  const int z1 = min(z0 + zchunk, nz);
  const int tid = threadIdx.x;
  for (int i = tid; i < kFP3; i += kFThreads) S.gx[i] = pmod(x0 - 2 + i, nx);
  for (int i = tid; i < kFTY + 4; i += kFThreads) S.gy[i] = pmod(y0 - 2 + i, ny) * nx;
  __syncthreads();

  const int64_t n3 = K.n3, npts = 2 * n3, plane = (int64_t)nx * ny;
  const int64_t sbase = (int64_t)s * n3;
  const Real E0 = K.E0, dt = K.dt;
  const Real t0d = K.delta * K.theta0;

  // Er* and v of plane k on the front region
  auto load_front = [&](int k) {
    const int64_t zo = sbase + (int64_t)pmod(k, nz) * plane;
    const int s2 = (k + 6) & 1, s3 = (k + 6) % 3;
    for (int i = tid; i < kFR3; i += kFThreads) {
      const int ly = i / kFP3, lx = i - ly * kFP3;
      const int64_t q = zo + S.gy[ly] + S.gx[lx];
      S.es[s2][i] = es_g[q];
      S.vx[s2][i] = vadv(ucur, uprev, q);
      S.vy[s2][i] = vadv(ucur, uprev, npts + q);
      S.vz[s3][i] = vadv(ucur, uprev, 2 * npts + q);
    }
  };
  // kappa_R and rho - 1 of plane k on the corrector region
  auto load_back = [&](int k) {
    const int64_t zo = sbase + (int64_t)pmod(k, nz) * plane;
    const int s4 = (k + 8) & 3;
    for (int i = tid; i < kFR1; i += kFThreads) {
      const int ly = i / kFP1, lx = i - ly * kFP1;
      const int64_t q = zo + S.gy[ly + 1] + S.gx[lx + 1];
      S.kap[s4][i] = kap_g[q];
      S.dr[i] = drho_g[q];
    }
  };

  load_front(z0 - 2);
  for (int k = z0 - 2; k <= z1; ++k) {
    load_front(k + 1);
    load_back(k);
    __syncthreads();
    // predictor of plane k (forward differences; +z from plane k+1)
    {
      const int a2 = (k + 6) & 1, n2 = (k + 7) & 1, a3 = (k + 6) % 3, n3s = (k + 7) % 3;
      const Real* es = S.es[a2];
      const Real* vx = S.vx[a2];
      const Real* vy = S.vy[a2];
      const Real* vz = S.vz[a3];
      Real* ep = S.ep[a2];
      for (int i = tid; i < kFR2; i += kFThreads) {
        const int ly = i / kFP2, lx = i - ly * kFP2;
        const int c = ly * kFP3 + lx;  // same origin (-2, -2) as the front region
        const Real e0 = es[c];
        Real div = Real(0);
        {
          const Real vp = vx[c], vq = vx[c + 1];
          div += E0 * (vq - vp) + (es[c + 1] * vq - e0 * vp);
        }
        {
          const Real vp = vy[c], vq = vy[c + kFP3];
          div += E0 * (vq - vp) + (es[c + kFP3] * vq - e0 * vp);
        }
        {
          const Real vp = vz[c], vq = S.vz[n3s][c];
          div += E0 * (vq - vp) + (S.es[n2][c] * vq - e0 * vp);
        }
        ep[i] = e0 - dt * div;
      }
    }
    __syncthreads();
    // corrector and theta_R of plane k (backward differences; -z from plane k-1)
    if (k >= z0 - 1) {
      const int a2 = (k + 6) & 1, p2 = (k + 5) & 1, a3 = (k + 6) % 3, p3 = (k + 5) % 3;
      const Real* es = S.es[a2];
      const Real* vx = S.vx[a2];
      const Real* vy = S.vy[a2];
      const Real* vz = S.vz[a3];
      const Real* vzm = S.vz[p3];
      const Real* ep = S.ep[a2];
      const Real* epm = S.ep[p2];
      Real* th = S.th[a3];
      Real* ec = S.ec[a2];
      for (int i = tid; i < kFR1; i += kFThreads) {
        const int ly = i / kFP1, lx = i - ly * kFP1;
        const int c2 = (ly + 1) * kFP2 + (lx + 1);
        const int c3 = (ly + 1) * kFP3 + (lx + 1);
        const Real epp = ep[c2];
        Real div = Real(0);
        {
          const Real vp = vx[c3], vq = vx[c3 - 1];
          div += E0 * (vp - vq) + (epp * vp - ep[c2 - 1] * vq);
        }
        {
          const Real vp = vy[c3], vq = vy[c3 - kFP3];
          div += E0 * (vp - vq) + (epp * vp - ep[c2 - kFP2] * vq);
        }
        {
          const Real vp = vz[c3], vq = vzm[c3];
          div += E0 * (vp - vq) + (epp * vp - epm[c2] * vq);
        }
        const Real val = Real(0.5) * (es[c3] + epp - dt * div);
        const Real dr = S.dr[i];
        th[i] = (Real(2) * val - t0d * dr) / (K.delta * (Real(1) + dr));
        const int tx_ = lx - 1, ty_ = ly - 1;
        if (tx_ >= 0 && tx_ < kFTX && ty_ >= 0 && ty_ < kFTY) ec[ty_ * kFTX + tx_] = val;
      }
    }
    __syncthreads();
    // first FTCS sub-step of plane k - 1 on the tile
    if (k >= z0 + 1) {
      const int zo = k - 1;
      const int m3 = (k + 5) % 3, l3 = (k + 4) % 3, h3 = (k + 6) % 3;
      const int m4 = (k + 7) & 3, l4 = (k + 6) & 3, h4 = (k + 8) & 3;
      const Real* th = S.th[m3];
      const Real* kp_ = S.kap[m4];
      const Real* ec = S.ec[(k + 5) & 1];
      const int64_t obase = sbase + (int64_t)pmod(zo, nz) * plane;
      for (int j = tid; j < kFT; j += kFThreads) {
        const int ly = j / kFTX, lx = j - ly * kFTX;
        if (x0 + lx >= nx || y0 + ly >= ny) continue;
        const int c = (ly + 1) * kFP1 + (lx + 1);
        const Real thp = th[c], kp = kp_[c];
        Real acc = Real(0);
        acc += Real(0.5) * (kp + kp_[c - 1]) * (th[c - 1] - thp);
        acc += Real(0.5) * (kp + kp_[c + 1]) * (th[c + 1] - thp);
        acc += Real(0.5) * (kp + kp_[c - kFP1]) * (th[c - kFP1] - thp);
        acc += Real(0.5) * (kp + kp_[c + kFP1]) * (th[c + kFP1] - thp);
        acc += Real(0.5) * (kp + S.kap[l4][c]) * (S.th[l3][c] - thp);
        acc += Real(0.5) * (kp + S.kap[h4][c]) * (S.th[h3][c] - thp);
        e_next[obase + (int64_t)(y0 + ly) * nx + (x0 + lx)] = ec[j] + K.hsub * acc;
      }
    }
  }
}

// z planes per block: enough blocks for about three waves of the resident
// blocks (blocks_per_sm x sms), at least 4 planes.
inline int fused_zchunk(int nx, int ny, int nz, int sms, int blocks_per_sm) {
  const int64_t tiles = (int64_t)((nx + kFTX - 1) / kFTX) * ((ny + kFTY - 1) / kFTY) * 2;
  const int64_t want = 3 * (int64_t)sms * blocks_per_sm;
  int64_t chunks = (want + tiles - 1) / tiles;
  if (chunks < 1) chunks = 1;
  int zc = (int)((nz + chunks - 1) / chunks);
  if (zc < 4) zc = 4;
  return zc;
}

}  // namespace rpk
