// Device helpers of the reduced polyatomic ES-BGK lattice-Boltzmann step
// (Kolluru, Atif & Ansumali, arXiv 2201.05280, Sec. 4 and Sec. 5): storage
// conversions, per-launch constants, moments, the f-level recovery, Hermite
// targets and the BCC pull gather.
//
// Data layout (HBM):
//   populations  Store pop[2][41][nz][ny][nx] per buffer, i.e. element
//                (s*41 + q)*n3 + (z*ny + y)*nx + x; two buffers ping-pong.
//                Reduced-precision storage holds h_q = g_q/w_q - 1; FP64 too.
//   scalar fields Real f[2][nz][ny][nx] (point index p = s*n3 + cell).
//   e            auxiliary rotational energy minus delta*theta0/2 (deviation)
//   drho         rho - 1 of the last collision
//   u            two ring slots of 3 planes each: u(t) and u(t-1)
//   kap          kappa_R of the last collision
// The state between steps is "post-collision, pre-stream": the collide kernel
// pulls g(x - c_q) from the previous buffer. Right after initialisation the
// state is post-stream instead (kPull = false reads the point's own slot).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <utility>

#include "rpk_lattice.cuh"
#include "rpk_vec2.cuh"

namespace rpk {

// ---------------------------------------------------------------------------
// storage conversions

template <typename S, typename R>
__device__ __forceinline__ R to_real(S v) { return static_cast<R>(v); }
template <>
__device__ __forceinline__ float to_real<__half, float>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_real<__nv_bfloat16, float>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <typename S, typename R>
__device__ __forceinline__ S from_real(R v) { return static_cast<S>(v); }
template <>
__device__ __forceinline__ __half from_real<__half, float>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_real<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}

// compile-time loop: f(std::integral_constant<int, K>) for K = 0..N-1
template <typename F, int... K>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, K...>) {
  (f(std::integral_constant<int, K>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------------------
// per-launch constants (host fills them in double, then casts)

template <typename Real>
struct StepConst {
  int nx, ny, nz;
  int64_t n3;     // nx*ny*nz
  Real theta0;
  Real c_keep;    // 1 - 2 beta*
  Real c_relax;   // 2 beta*
  Real beta;      // beta* = dt/(2 tau* + dt)
  Real w_es;      // tau*/tau
  Real w_eq;      // tau*/tau1
  Real b;
  Real inv_sig;   // 1 / (1 + dt/(2 tau*) - b dt/(2 tau))
  Real inv_d;     // 1 / (1 + dt/(2 tau1))
  Real delta;
  Real inv_3pd;   // 1 / (3 + delta)
  Real exc;       // dt delta / (2 tau1)
  Real kapc;      // k_r 5 tau / (2 B), kappa_R = kapc * rho * theta
  Real E0;        // delta theta0 / 2
  Real dt;
  Real hsub;      // dt / nsub
  // paper mode of the rotational solver (Sec. 5, four steps on theta_R):
  int paper;      // 1: the state holds theta_R - theta0 instead of the auxiliary energy
  Real ra_keep;   // 1 / (1 + X), X = 3 dt / (2 tau1 (3 + delta)): backward-Euler half step
  Real ra_t;      // X / (1 + X)
  Real pa;        // a = delta X / 3: theta_T(g) = theta_T + a (theta_T - theta_R)
  Real inv_1pa;   // 1 / (1 + a)
};

// Ghost values, one block of kGhostStride per x end (reservoirs, blocks 0, 1)
// or per wall (low / high y wall in blocks 0, 1, low / high x wall in blocks
// 2, 3: h of f^eq(1, u_w, theta_w), its e, rho - 1 = 0, u_w, kappa_R).
constexpr int kGhostStride = 48;
constexpr int kGhostBlocks = 4;

// Boundary kinds of the templated kernels (kBC): 0 periodic; 1 x reservoirs;
// otherwise a mask of diffuse walls, kWallY normal to y and kWallX normal to x.
constexpr int kWallY = 2, kWallX = 4;
enum { kGhE = 41, kGhDrho = 42, kGhU = 43, kGhKap = 46 };

// ---------------------------------------------------------------------------
// moments and Hermite targets (all in deviation form about rho = 1, theta0)

template <typename Real>
struct Mom {
  Real drho, rho, inv_rho;
  Real j[3];
  Real dP[6];    // sum w h c_a c_b: xx yy zz xy xz yz
  Real dTg;      // theta_T(g) - theta0
  Real dth;      // theta - theta0 (eq. thetadef)
  Real dT, dR;   // theta_T(f) - theta0, theta_R - theta0
  Real sig[6];   // sigma(f), a density
};

// rho, j, P of g = w (1 + h), pair by pair. Generic over the value type V
// (float, double, or F2 = the same quantity at two points).
template <typename V>
__device__ __forceinline__ void raw_moments(const V (&h)[kQ], Mom<V>& m) {
  using S = scalar_t<V>;
  V d = S(kWeightRest) * h[0];
  V jx = splat<V>(0), jy = jx, jz = jx, pxx = jx, pyy = jx, pzz = jx, pxy = jx, pxz = jx, pyz = jx;
  static_for<kPairs>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr Vel2 v = kPairVel2[k];
    constexpr double w = pair_weight(k);
    const V ev = S(w) * (h[2 * k + 1] + h[2 * k + 2]);
    const V od = S(w) * (h[2 * k + 1] - h[2 * k + 2]);
    d += ev;
    if constexpr (v.x != 0) jx = fmad(S(0.5 * v.x), od, jx);
    if constexpr (v.y != 0) jy = fmad(S(0.5 * v.y), od, jy);
    if constexpr (v.z != 0) jz = fmad(S(0.5 * v.z), od, jz);
    if constexpr (v.x != 0) pxx = fmad(S(0.25 * v.x * v.x), ev, pxx);
    if constexpr (v.y != 0) pyy = fmad(S(0.25 * v.y * v.y), ev, pyy);
    if constexpr (v.z != 0) pzz = fmad(S(0.25 * v.z * v.z), ev, pzz);
    if constexpr (v.x * v.y != 0) pxy = fmad(S(0.25 * v.x * v.y), ev, pxy);
    if constexpr (v.x * v.z != 0) pxz = fmad(S(0.25 * v.x * v.z), ev, pxz);
    if constexpr (v.y * v.z != 0) pyz = fmad(S(0.25 * v.y * v.z), ev, pyz);
  });
  m.drho = d;
  m.rho = S(1) + d;
  m.inv_rho = S(1) / m.rho;
  m.j[0] = jx; m.j[1] = jy; m.j[2] = jz;
  m.dP[0] = pxx; m.dP[1] = pyy; m.dP[2] = pzz;
  m.dP[3] = pxy; m.dP[4] = pxz; m.dP[5] = pyz;
}

// f-level moments from g (Sec. 5, g/f relations) and the stored auxiliary
// rotational energy e (deviation) -- or, in paper mode, the stored theta_R:
// then theta_T(f) = (theta_T(g) + a theta_R)/(1 + a) inverts the printed
// theta_T(g) relation.
//   theta_T(g) = (tr P - j^2/rho)/(3 rho)
//   Rt = 2 Er/(delta rho)  (auxiliary rotational temperature)
//   theta = (3 theta_T(g) + delta Rt)/(3 + delta)   (invariant of the transform)
//   D = (theta_T(g) - Rt)/(1 + dt/(2 tau1)) = theta_T(f) - theta_R
//   theta_T(f) = theta + delta D/(3 + delta),  theta_R = theta - 3 D/(3 + delta)
//   sigma(f) = (P - jj/rho - rho theta_T(g) I)/(1 + dt/(2 tau*) - b dt/(2 tau))
template <typename Real, bool kPaper = false, typename V>
__device__ __forceinline__ void recover(Mom<V>& m, V e, const StepConst<Real>& K) {
  using S = scalar_t<V>;
  const S t0 = K.theta0;
  const V jj = fmad(m.j[2], m.j[2], fmad(m.j[1], m.j[1], m.j[0] * m.j[0]));
  const V trdP = m.dP[0] + m.dP[1] + m.dP[2];
  m.dTg = (trdP - jj * m.inv_rho - S(3) * t0 * m.drho) * m.inv_rho * S(1.0 / 3.0);
  if constexpr (kPaper) {
    // paper mode: e is theta_R - theta0 itself
    m.dR = e;
    m.dT = fmad(K.pa, m.dR, m.dTg) * K.inv_1pa;
    m.dth = fmad(K.delta, m.dR, S(3) * m.dT) * K.inv_3pd;
  } else {
    const V dRt = (S(2) * e - K.delta * t0 * m.drho) * m.inv_rho / K.delta;
    m.dth = fmad(K.delta, dRt, S(3) * m.dTg) * K.inv_3pd;
    const V D = (m.dTg - dRt) * K.inv_d;
    m.dT = fmad(K.delta * K.inv_3pd, D, m.dth);
    m.dR = m.dth - (S(3) * K.inv_3pd) * D;
  }
  const V iso = fmad(t0, m.drho, m.rho * m.dTg);
  const V ir = m.inv_rho;
  m.sig[0] = (m.dP[0] - m.j[0] * m.j[0] * ir - iso) * K.inv_sig;
  m.sig[1] = (m.dP[1] - m.j[1] * m.j[1] * ir - iso) * K.inv_sig;
  m.sig[2] = (m.dP[2] - m.j[2] * m.j[2] * ir - iso) * K.inv_sig;
  m.sig[3] = (m.dP[3] - m.j[0] * m.j[1] * ir) * K.inv_sig;
  m.sig[4] = (m.dP[4] - m.j[0] * m.j[2] * ir) * K.inv_sig;
  m.sig[5] = (m.dP[5] - m.j[1] * m.j[2] * ir) * K.inv_sig;
}

// Coefficients of f_q/w_q - 1 for the third-order Hermite expansion of a
// Gaussian (rho, u, Lambda) about the lattice weights; Dl = Lambda - theta0 I.
//   f/w = rho + j.c/t0 + A2:(cc - t0 I)/(2 t0^2) + A3:H3(c)/(6 t0^3)
//   A2 = jj/rho + rho Dl,  A3_abc = j_a j_b j_c/rho^2 + Dl_ab j_c + Dl_bc j_a + Dl_ca j_b
// even part: e0 + sum E_ab c_a c_b ; odd part: sum O_a c_a + cubic terms.
template <typename Real>
struct Herm {
  Real e0, exx, eyy, ezz, exy, exz, eyz;
  Real ox, oy, oz;
  Real oxxx, oyyy, ozzz, oxxy, oxxz, oyyx, oyyz, ozzx, ozzy, oxyz;
};

template <typename V>
__device__ __forceinline__ void hermite(V drho, V rho, V inv_rho, const V (&j)[3], const V (&Dl)[6],
                                        scalar_t<V> t0, Herm<V>& H) {
  using S = scalar_t<V>;
  const V jx = j[0], jy = j[1], jz = j[2];
  const V jxr = jx * inv_rho, jyr = jy * inv_rho, jzr = jz * inv_rho;
  const V a2xx = fmad(jx, jxr, rho * Dl[0]);
  const V a2yy = fmad(jy, jyr, rho * Dl[1]);
  const V a2zz = fmad(jz, jzr, rho * Dl[2]);
  const V a2xy = fmad(jx, jyr, rho * Dl[3]);
  const V a2xz = fmad(jx, jzr, rho * Dl[4]);
  const V a2yz = fmad(jy, jzr, rho * Dl[5]);
  // j_a j_b j_c / rho^2 = (j_a j_b / rho)(j_c / rho)
  const V xx = jx * jxr, yy = jy * jyr, zz = jz * jzr;
  const V dxx = Dl[0], dyy = Dl[1], dzz = Dl[2], dxy = Dl[3], dxz = Dl[4], dyz = Dl[5];
  const V a3xxx = fmad(S(3) * dxx, jx, xx * jxr);
  const V a3yyy = fmad(S(3) * dyy, jy, yy * jyr);
  const V a3zzz = fmad(S(3) * dzz, jz, zz * jzr);
  const V a3xxy = fmad(dxx, jy, fmad(S(2) * dxy, jx, xx * jyr));
  const V a3xxz = fmad(dxx, jz, fmad(S(2) * dxz, jx, xx * jzr));
  const V a3yyx = fmad(dyy, jx, fmad(S(2) * dxy, jy, yy * jxr));
  const V a3yyz = fmad(dyy, jz, fmad(S(2) * dyz, jy, yy * jzr));
  const V a3zzx = fmad(dzz, jx, fmad(S(2) * dxz, jz, zz * jxr));
  const V a3zzy = fmad(dzz, jy, fmad(S(2) * dyz, jz, zz * jyr));
  const V a3xyz = fmad(dxy, jz, fmad(dyz, jx, fmad(dxz, jy, (jx * jyr) * jzr)));
  const S i1 = S(1) / t0;
  const S i2 = i1 * i1;
  const S i3 = i2 * i1;
  // even part
  H.e0 = drho - (S(0.5) * i1) * (a2xx + a2yy + a2zz);
  H.exx = (S(0.5) * i2) * a2xx;
  H.eyy = (S(0.5) * i2) * a2yy;
  H.ezz = (S(0.5) * i2) * a2zz;
  H.exy = i2 * a2xy;
  H.exz = i2 * a2xz;
  H.eyz = i2 * a2yz;
  // odd part: j.c/t0 - t0 * 3 V.c/(6 t0^3), V_a = sum_b A3_abb
  const V vx = a3xxx + a3yyx + a3zzx;
  const V vy = a3xxy + a3yyy + a3zzy;
  const V vz = a3xxz + a3yyz + a3zzz;
  H.ox = fmad(-S(0.5) * i2, vx, jx * i1);
  H.oy = fmad(-S(0.5) * i2, vy, jy * i1);
  H.oz = fmad(-S(0.5) * i2, vz, jz * i1);
  const S s6 = i3 * S(1.0 / 6.0), s2 = i3 * S(0.5);
  H.oxxx = s6 * a3xxx;
  H.oyyy = s6 * a3yyy;
  H.ozzz = s6 * a3zzz;
  H.oxxy = s2 * a3xxy;
  H.oxxz = s2 * a3xxz;
  H.oyyx = s2 * a3yyx;
  H.oyyz = s2 * a3yyz;
  H.ozzx = s2 * a3zzx;
  H.ozzy = s2 * a3zzy;
  H.oxyz = i3 * a3xyz;
}

template <int VX, int VY, int VZ, typename V>
__device__ __forceinline__ V herm_even(const Herm<V>& H) {
  using S = scalar_t<V>;
  constexpr double cx = 0.5 * VX, cy = 0.5 * VY, cz = 0.5 * VZ;
  V r = H.e0;
  if constexpr (VX != 0) r = fmad(S(cx * cx), H.exx, r);
  if constexpr (VY != 0) r = fmad(S(cy * cy), H.eyy, r);
  if constexpr (VZ != 0) r = fmad(S(cz * cz), H.ezz, r);
  if constexpr (VX * VY != 0) r = fmad(S(cx * cy), H.exy, r);
  if constexpr (VX * VZ != 0) r = fmad(S(cx * cz), H.exz, r);
  if constexpr (VY * VZ != 0) r = fmad(S(cy * cz), H.eyz, r);
  return r;
}

template <int VX, int VY, int VZ, typename V>
__device__ __forceinline__ V herm_odd(const Herm<V>& H) {
  using S = scalar_t<V>;
  constexpr double cx = 0.5 * VX, cy = 0.5 * VY, cz = 0.5 * VZ;
  V r = splat<V>(0);
  if constexpr (VX != 0) r = fmad(S(cx * cx * cx), H.oxxx, fmad(S(cx), H.ox, r));
  if constexpr (VY != 0) r = fmad(S(cy * cy * cy), H.oyyy, fmad(S(cy), H.oy, r));
  if constexpr (VZ != 0) r = fmad(S(cz * cz * cz), H.ozzz, fmad(S(cz), H.oz, r));
  if constexpr (VX * VY != 0) r = fmad(S(cy * cy * cx), H.oyyx, fmad(S(cx * cx * cy), H.oxxy, r));
  if constexpr (VX * VZ != 0) r = fmad(S(cz * cz * cx), H.ozzx, fmad(S(cx * cx * cz), H.oxxz, r));
  if constexpr (VY * VZ != 0) r = fmad(S(cz * cz * cy), H.ozzy, fmad(S(cy * cy * cz), H.oyyz, r));
  if constexpr (VX * VY * VZ != 0) r = fmad(S(cx * cy * cz), H.oxyz, r);
  return r;
}

// Hermite coefficients of f^mix = tau*(f^ES/tau + f^Eq/tau1) (Sec. 5): both
// targets share rho and u and are linear in Lambda, so
//   Lambda_mix = (tau*/tau)(theta_T I + b sigma/rho) + (tau*/tau1) theta I.
template <typename Real, typename V>
__device__ __forceinline__ void mix_coeffs(const Mom<V>& m, const StepConst<Real>& K, Herm<V>& H) {
  const V iso = fmad(K.w_eq, m.dth, K.w_es * m.dT);
  const V bs = (K.w_es * K.b) * m.inv_rho;
  V Dl[6] = {fmad(bs, m.sig[0], iso), fmad(bs, m.sig[1], iso), fmad(bs, m.sig[2], iso),
             bs * m.sig[3], bs * m.sig[4], bs * m.sig[5]};
  hermite(m.drho, m.rho, m.inv_rho, m.j, Dl, K.theta0, H);
}

// ---------------------------------------------------------------------------
// geometry helpers

__device__ __forceinline__ int wrap_near(int a, int n) {
  // valid for |a - [0, n)| <= 2; n == 1 maps everything to 0
  return n == 1 ? 0 : (a < 0 ? a + n : (a >= n ? a - n : a));
}

struct PointIdx {
  int s, x, y, z;
  int64_t cell;  // (z*ny + y)*nx + x
};

template <typename Real>
__device__ __forceinline__ bool point_from_block(const StepConst<Real>& K, PointIdx& P) {
  P.x = blockIdx.x * blockDim.x + threadIdx.x;
  P.y = blockIdx.y;
  P.s = blockIdx.z / K.nz;
  P.z = blockIdx.z - P.s * K.nz;
  if (P.x >= K.nx) return false;
  P.cell = ((int64_t)P.z * K.ny + P.y) * K.nx + P.x;
  return true;
}

// Gather the 41 populations of point P: from its own slots (kPull = false) or
// pulled from x - c_q (kPull = true; Sec. 5, BCC layout: a half velocity
// from sublattice 0 at index x comes from sublattice 1 at x - (c > 0 ? 1 : 0)
// per axis, and from sublattice 1 it comes from sublattice 0 at
// x + (c < 0 ? 1 : 0)). kBC = 1: sources beyond the x ends read the reservoir.
// kBC & kWallY: sources beyond a y wall (y = -1/4, y = ny - 1/4) are emitted by
// the wall, g = rho_w f^eq(1, u_w, theta_w), i.e. h = d + hw + d hw with
// d = rho_w - 1 of the point's (x, z) column (wcol[(wall * nz + z) * nx + x])
// and hw the wall's table entry. kBC & kWallX: the same for the x walls
// (x = -1/4, x = nx - 1/4) with the (y, z) columns at
// wcol[2 nx nz + (wall * nz + z) * ny + y]; a source beyond both a y and an x
// wall belongs to the y wall.
template <typename Store, typename Real, bool kPull, int kBC>
__device__ __forceinline__ void gather(const Store* __restrict__ pin,
                                       const Real* __restrict__ ghost, const StepConst<Real>& K,
                                       const PointIdx& P, Real (&h)[kQ],
                                       const Real* __restrict__ wcol = nullptr) {
  const int64_t n3 = K.n3;
  if constexpr (!kPull) {
    const Store* base = pin + (int64_t)(P.s * kQ) * n3 + P.cell;
#pragma unroll
    for (int q = 0; q < kQ; ++q) h[q] = to_real<Store, Real>(base[(int64_t)q * n3]);
  } else {
    const int nx = K.nx, ny = K.ny, nz = K.nz;
    int xw[5], yw[5], zw[5];
    bool xin[5], yin[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      xw[k] = wrap_near(P.x + k - 2, nx);
      yw[k] = wrap_near(P.y + k - 2, ny);
      zw[k] = wrap_near(P.z + k - 2, nz);
      xin[k] = (P.x + k - 2 >= 0) && (P.x + k - 2 < nx);
      yin[k] = (P.y + k - 2 >= 0) && (P.y + k - 2 < ny);
    }
    // half-velocity source offsets: c > 0 -> s - 1, c < 0 -> s
    const int s = P.s;
    const int xhp = s ? xw[2] : xw[1], xhm = s ? xw[3] : xw[2];
    const int yhp = s ? yw[2] : yw[1], yhm = s ? yw[3] : yw[2];
    const int zhp = s ? zw[2] : zw[1], zhm = s ? zw[3] : zw[2];
    const bool xinhp = s ? xin[2] : xin[1], xinhm = s ? xin[3] : xin[2];
    const bool yinhp = s ? yin[2] : yin[1], yinhm = s ? yin[3] : yin[2];
    const Store* same = pin + (int64_t)(s * kQ) * n3;
    const Store* other = pin + (int64_t)((1 - s) * kQ) * n3;
    h[0] = to_real<Store, Real>(same[P.cell]);
    static_for<kQ - 1>([&](auto qc) {
      constexpr int q = decltype(qc)::value + 1;
      constexpr Vel2 v = vel2(q);
      constexpr bool half = (v.x & 1) != 0;
      int xs, ys, zs;
      [[maybe_unused]] bool insx = true, insy = true;
      const Store* base;
      if constexpr (half) {
        xs = v.x > 0 ? xhp : xhm;
        ys = v.y > 0 ? yhp : yhm;
        zs = v.z > 0 ? zhp : zhm;
        insx = v.x > 0 ? xinhp : xinhm;
        insy = v.y > 0 ? yinhp : yinhm;
        base = other;
      } else {
        xs = xw[2 - v.x / 2];
        ys = yw[2 - v.y / 2];
        zs = zw[2 - v.z / 2];
        insx = xin[2 - v.x / 2];
        insy = yin[2 - v.y / 2];
        base = same;
      }
      const int64_t cell = ((int64_t)zs * ny + ys) * nx + xs;
      if constexpr (kBC == 1) {
        if (!insx) {
          h[q] = ghost[(v.x > 0 ? 0 : kGhostStride) + q];
          return;
        }
      }
      if constexpr ((kBC & kWallY) && v.y != 0) {
        if (!insy) {
          const int w = v.y > 0 ? 0 : 1;  // source below the low wall / above the high wall
          const Real d = wcol[((int64_t)w * nz + P.z) * nx + P.x];
          const Real hw = ghost[w * kGhostStride + q];
          h[q] = d + hw + d * hw;
          return;
        }
      }
      if constexpr ((kBC & kWallX) && v.x != 0) {
        if (!insx) {
          const int w = v.x > 0 ? 0 : 1;
          const Real d = wcol[2 * (int64_t)nx * nz + ((int64_t)w * nz + P.z) * ny + P.y];
          const Real hw = ghost[(2 + w) * kGhostStride + q];
          h[q] = d + hw + d * hw;
          return;
        }
      }
      h[q] = to_real<Store, Real>(base[(int64_t)q * n3 + cell]);
    });
  }
}

// rho_w - 1 of every wall column, from the post-collision populations pin that
// the next pull reads. For a wall and one of its columns: the column's
// populations whose destination lies beyond the wall carry the mass
// M_out = sum w (1 + h); the wall emits rho_w f^eq(1, u_w, theta_w) into the
// column's entries whose source lies beyond it, mass rho_w D with
// D = sum w (1 + hw). rho_w - 1 = (M_out - D) / D, accumulated as
// (sum_out w - sum_in w) + sum_out w h - sum_in w hw so that the deviation keeps
// its precision (the weights of c and -c are equal). A velocity with |2 c_a| = n
// along the wall normal a has its n layers next to the wall in play. Where
// both kinds of walls are on, a population crossing a y wall belongs to it
// even if it crosses an x wall too, so the x walls count only entries whose
// other end stays inside in y.
// One thread per (wall, column): y walls first (slots [0, 2 nx nz), columns
// (x, z)), then x walls (slots 2 nx nz + [0, 2 ny nz), columns (y, z)).
template <typename Store, typename Real, int kBC>
__global__ void __launch_bounds__(128)
    k_wall_rho(StepConst<Real> K, const Store* __restrict__ pin, const Real* __restrict__ ghost,
               Real* __restrict__ wcol) {
  const int64_t ny_cols = (int64_t)K.nx * K.nz, nx_cols = (int64_t)K.ny * K.nz;
  const int64_t ybase = (kBC & kWallY) ? 2 * ny_cols : 0;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ybase + ((kBC & kWallX) ? 2 * nx_cols : 0)) return;
  const bool xwall = t >= ybase;
  int64_t slot = t;
  if (xwall) {
    t -= ybase;
    slot = 2 * ny_cols + t;
  }
  const int64_t ncol = xwall ? nx_cols : ny_cols;
  const int w = t >= ncol ? 1 : 0;
  const int64_t c = t - w * ncol;
  const int nx = K.nx, ny = K.ny;
  // column coordinates: (x, z) for a y wall, (y, z) for an x wall
  const int ca = (int)(c % (xwall ? ny : nx)), z = (int)(c / (xwall ? ny : nx));
  const int nn = xwall ? nx : ny;  // cells along the wall normal
  const int64_t n3 = K.n3;
  const Real* hw = ghost + ((xwall ? 2 : 0) + w) * kGhostStride;
  Real base = Real(0), A = Real(0), D = Real(0), S = Real(0);
  static_for<kQ - 1>([&](auto qc) {
    constexpr int q = decltype(qc)::value + 1;
    constexpr Vel2 v = vel2(q);
    const int vn = xwall ? v.x : v.y;  // doubled velocity along the normal
    const int vt = xwall ? v.y : 0;    // along y, for the corner rule of the x walls
    if (vn == 0) return;
    const int n = vn > 0 ? vn : -vn;
    const Real wq = Real(weight(q));
    const bool emitted = (w == 0) == (vn > 0);
    for (int k = 0; k < n; ++k) {
      const int L2 = w == 0 ? k : 2 * nn - 1 - k;  // 2 * index + s along the normal
      const int s = L2 & 1, i = L2 >> 1;
      if ((kBC & kWallY) && xwall) {
        // the other end of the trajectory must stay inside in y
        const int Y2 = 2 * ca + s + (emitted ? -vt : vt);
        if (Y2 < 0 || Y2 >= 2 * ny) continue;
      }
      if (emitted) {
        D += wq * (Real(1) + hw[q]);
        A -= wq * hw[q];
        base -= wq;
      } else {
        const int x = xwall ? i : ca, y = xwall ? ca : i;
        S += wq * to_real<Store, Real>(pin[(int64_t)(s * kQ + q) * n3 + ((int64_t)z * ny + y) * nx + x]);
        base += wq;
      }
    }
  });
  wcol[slot] = (base + A + S) / D;
}

}  // namespace rpk
