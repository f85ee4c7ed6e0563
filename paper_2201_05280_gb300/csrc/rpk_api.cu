// C-ABI layer of librpk: the lattice object, parameter mapping, validation,
// host<->device staging and checkpoints. See include/rpk.h for the contract of
// every entry point. Kernels are launched through rpk::Ops<Store, Real>.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rpk_internal.h"
#include "rpk_kernels.cuh"

namespace rpk {

extern template struct Ops<double, double>;
extern template struct Ops<float, float>;
extern template struct Ops<__half, float>;
extern template struct Ops<__nv_bfloat16, float>;

static thread_local std::string g_error;

void set_error(const std::string& msg) { g_error = msg; }

rpk_status cuda_fail(cudaError_t err, const char* what) {
  set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(err));
  return RPK_ERR_CUDA;
}

rpk_status fail(rpk_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

// Dispatch on the storage precision.
template <typename F>
static rpk_status with_ops(int precision, F&& f) {
  switch (precision) {
    case RPK_F64: return f(Ops<double, double>{});
    case RPK_F32: return f(Ops<float, float>{});
    case RPK_F16DEV: return f(Ops<__half, float>{});
    case RPK_BF16DEV: return f(Ops<__nv_bfloat16, float>{});
    default: return fail(RPK_ERR_ARG, "unknown precision");
  }
}

rpk_status validate_relax(const rpk_relax* r) {
  if (!r) return fail(RPK_ERR_ARG, "relax is NULL");
  if (!(r->delta > 0.0) || !std::isfinite(r->delta)) return fail(RPK_ERR_PARAM, "delta must be > 0");
  if (!(r->tau > 0.0) || !std::isfinite(r->tau)) return fail(RPK_ERR_PARAM, "tau must be > 0");
  if (!(r->tau1 > 0.0) || !std::isfinite(r->tau1)) return fail(RPK_ERR_PARAM, "tau1 must be > 0");
  if (!(r->k_r >= 0.0) || !std::isfinite(r->k_r)) return fail(RPK_ERR_PARAM, "k_r must be >= 0");
  if (!std::isfinite(r->b)) return fail(RPK_ERR_PARAM, "b must be finite");
  const double B = 1.0 + r->tau / r->tau1;
  if (!(B - r->b > 0.0)) return fail(RPK_ERR_PARAM, "B - b must be > 0 (B = 1 + tau/tau1)");
  if (r->dt != 1.0) return fail(RPK_ERR_PARAM, "dt must be 1 in lattice units");
  if (r->nsub < 0 || r->nsub > 4096) return fail(RPK_ERR_PARAM, "nsub must lie in [0, 4096]");
  return RPK_OK;
}

cudaError_t timing_begin(rpk_lattice* L) {
  if (!L->timing) return cudaSuccess;
  const size_t need = 2 * (L->ev_used + 1);
  while (L->events.size() < need) {
    cudaEvent_t ev;
    cudaError_t err = cudaEventCreate(&ev);
    if (err != cudaSuccess) return err;
    L->events.push_back(ev);
  }
  return cudaEventRecord(L->events[2 * L->ev_used], L->stream);
}

cudaError_t timing_end(rpk_lattice* L, int cls, int kernels) {
  if (!L->timing) return cudaSuccess;
  cudaError_t err = cudaEventRecord(L->events[2 * L->ev_used + 1], L->stream);
  if (err != cudaSuccess) return err;
  if (L->ev_class.size() <= L->ev_used) {
    L->ev_class.resize(L->ev_used + 1);
    L->ev_kernels.resize(L->ev_used + 1);
  }
  L->ev_class[L->ev_used] = cls;
  L->ev_kernels[L->ev_used] = kernels;
  L->ev_used += 1;
  return cudaSuccess;
}

static int active_dims(const rpk_grid& g) {
  return (g.nx > 1) + (g.ny > 1) + (g.nz > 1);
}

}  // namespace rpk

using namespace rpk;

extern "C" {

int rpk_abi_version(void) { return RPK_ABI_VERSION; }

double rpk_theta0(void) { return kTheta0; }

const char* rpk_last_error(void) { return g_error.c_str(); }

rpk_status rpk_map_gas(double gamma, double eta, double eta_B, double kappa, double b,
                       double rho0, rpk_relax* out) {
  if (!out) return fail(RPK_ERR_ARG, "out is NULL");
  if (!(gamma > 1.0) || !(gamma <= 5.0 / 3.0)) return fail(RPK_ERR_PARAM, "gamma must lie in (1, 5/3]");
  if (!(eta > 0.0) || !(eta_B > 0.0) || !(kappa > 0.0) || !(rho0 > 0.0))
    return fail(RPK_ERR_PARAM, "eta, eta_B, kappa and rho0 must be > 0");
  const double delta = (5.0 - 3.0 * gamma) / (gamma - 1.0);
  if (!(delta > 0.0)) return fail(RPK_ERR_PARAM, "gamma = 5/3 leaves no rotational degrees of freedom");
  const double p0 = rho0 * kTheta0;
  const double c = 2.0 * delta / (3.0 * (3.0 + delta));
  const double tau1 = eta_B / (c * p0);
  const double denom = p0 - eta / tau1;
  const double tau = eta * (1.0 - b) / denom;
  if (!(denom != 0.0) || !(tau > 0.0) || !std::isfinite(tau))
    return fail(RPK_ERR_PARAM, "no tau > 0 for this eta_B/eta and b (eta_B/eta < 2 delta/(3(3+delta)) needs b > 1)");
  const double B = 1.0 + tau / tau1;
  const double kT = 5.0 * p0 * tau / (2.0 * B);
  double kr = kappa / kT - 1.0;
  if (kr < -1e-12) return fail(RPK_ERR_PARAM, "kappa below the translational conductivity: k_r < 0");
  if (kr < 0.0) kr = 0.0;
  out->delta = delta;
  out->tau = tau;
  out->tau1 = tau1;
  out->b = b;
  out->k_r = kr;
  out->dt = 1.0;
  out->nsub = 0;
  return validate_relax(out);
}

// FTCS sub-steps for a diffusion number D per sub-step with `diag` times D on
// the diagonal of the explicit update (2 ndim in the interior).
static int nsub_for_diagonal(const rpk_relax* r, double theta_max, double diag) {
  if (!r || !(r->k_r > 0.0) || !(diag > 0.0) || !(theta_max > 0.0)) return 1;
  const double B = 1.0 + r->tau / r->tau1;
  const double D = 5.0 * r->k_r * r->tau * (1.25 * theta_max) / (r->delta * B);
  const double n = std::ceil(diag * D * r->dt / 0.9);
  return (int)std::max(1.0, std::min(n, 4096.0));
}

int rpk_auto_nsub(const rpk_relax* r, double theta_max, int ndim) {
  if (ndim <= 0) return 1;
  return nsub_for_diagonal(r, theta_max, 2.0 * ndim);
}

rpk_status rpk_gas_from_nondim(double gamma, double nu, double lam, double Pr, double rho0,
                               double out[3]) {
  if (!out) return fail(RPK_ERR_ARG, "out is NULL");
  if (!(gamma > 1.0) || !(gamma <= 5.0 / 3.0)) return fail(RPK_ERR_PARAM, "gamma must lie in (1, 5/3]");
  if (!(nu > 0.0) || !(lam > 0.0) || !(Pr > 0.0) || !(rho0 > 0.0) || !std::isfinite(nu) ||
      !std::isfinite(lam) || !std::isfinite(Pr) || !std::isfinite(rho0))
    return fail(RPK_ERR_PARAM, "nu, eta_B/eta, Pr and rho0 must be finite and > 0");
  const double delta = (5.0 - 3.0 * gamma) / (gamma - 1.0);
  const double cp = 0.5 * (5.0 + delta);  // heat capacity per unit mass (theta units)
  const double eta = rho0 * nu;
  out[0] = eta;
  out[1] = lam * eta;
  out[2] = eta * cp / Pr;
  return RPK_OK;
}

double rpk_sound_speed(double gamma) {
  if (!(gamma > 1.0) || !(gamma <= 5.0 / 3.0)) return NAN;
  return std::sqrt(gamma * kTheta0);
}

int rpk_auto_nsub_fields(const rpk_relax* r, const double* theta_T, const double* theta_R,
                         int64_t n, const double* res, int ndim) {
  if (!r || (n > 0 && (!theta_T || !theta_R))) return 1;
  double tmax = 0.0;
  auto theta = [&](double T, double R) { return (3.0 * T + r->delta * R) / (3.0 + r->delta); };
  for (int64_t p = 0; p < n; ++p) tmax = std::max(tmax, theta(theta_T[p], theta_R[p]));
  if (res) tmax = std::max(tmax, std::max(theta(res[4], res[5]), theta(res[10], res[11])));
  if (!(tmax > 0.0) || !std::isfinite(tmax)) return 1;
  return rpk_auto_nsub(r, tmax, ndim);
}

static void free_all(rpk_lattice* L) {
  if (!L) return;
  for (cudaEvent_t ev : L->events) cudaEventDestroy(ev);
  L->events.clear();
  void* ptrs[] = {L->pop[0], L->pop[1], L->e,       L->e_star, L->e_a,    L->e_b,
                  L->vbuf,   L->thbuf,  L->drho,    L->kap,    L->u[0],   L->u[1],
                  L->ghost,  L->status, L->diag_partial, L->diag_out, L->stage, L->wrho};
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != L->device) cudaSetDevice(L->device);
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (prev >= 0 && prev != L->device) cudaSetDevice(prev);
}

rpk_status rpk_create(const rpk_grid* grid, void* cuda_stream, rpk_lattice** out) {
  if (!grid || !out) return fail(RPK_ERR_ARG, "grid or out is NULL");
  *out = nullptr;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(RPK_ERR_ARG, "nx, ny, nz must be >= 1");
  if (grid->ny > 65535 || 2 * (int64_t)grid->nz > 65535)
    return fail(RPK_ERR_ARG, "ny must be <= 65535 and nz <= 32767");
  if ((int64_t)grid->nx * grid->ny * grid->nz > (int64_t)1 << 31)
    return fail(RPK_ERR_ARG, "more than 2^31 cells per sublattice");
  if (grid->precision < RPK_F64 || grid->precision > RPK_BF16DEV) return fail(RPK_ERR_ARG, "bad precision");
  if (grid->bc_x != RPK_BC_PERIODIC && grid->bc_x != RPK_BC_RESERVOIR) return fail(RPK_ERR_ARG, "bad bc_x");
  rpk_lattice* L = new (std::nothrow) rpk_lattice();
  if (!L) return fail(RPK_ERR_OOM, "host allocation failed");
  L->grid = *grid;
  L->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t err = cudaGetDevice(&L->device);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&L->sms, cudaDevAttrMultiProcessorCount, L->device);
  if (err != cudaSuccess) {
    delete L;
    return cuda_fail(err, "cudaGetDevice");
  }
  L->n3 = (int64_t)grid->nx * grid->ny * grid->nz;
  L->npts = 2 * L->n3;
  L->real_elem = grid->precision == RPK_F64 ? sizeof(double) : sizeof(float);
  L->store_elem = grid->precision == RPK_F64 ? 8 : grid->precision == RPK_F32 ? 4 : 2;
  struct Req {
    void** p;
    size_t bytes;
  };
  const size_t popb = (size_t)kQ * L->npts * L->store_elem;
  const size_t fb = (size_t)L->npts * L->real_elem;
  Req reqs[] = {{&L->pop[0], popb}, {&L->pop[1], popb}, {&L->e, fb}, {&L->e_star, fb},
                {&L->e_a, fb}, {&L->e_b, fb}, {&L->vbuf, 3 * fb}, {&L->thbuf, fb},
                {&L->drho, fb}, {&L->kap, fb},
                {&L->u[0], 3 * fb}, {&L->u[1], 3 * fb},
                {&L->ghost, kGhostBlocks * kGhostStride * L->real_elem},
                {&L->wrho, (2 * (size_t)grid->nx * grid->nz + 2 * (size_t)grid->ny * grid->nz) * L->real_elem},
                {(void**)&L->status, sizeof(unsigned)},
                {(void**)&L->diag_partial, sizeof(double) * kDiagVals * kDiagBlocks},
                {(void**)&L->diag_out, sizeof(double) * 16}};
  for (auto& r : reqs) {
    err = cudaMalloc(r.p, r.bytes);
    if (err != cudaSuccess) {
      free_all(L);
      delete L;
      cudaGetLastError();
      return fail(err == cudaErrorMemoryAllocation ? RPK_ERR_OOM : RPK_ERR_CUDA,
                  std::string("device allocation failed: ") + cudaGetErrorString(err));
    }
    L->bytes_held += r.bytes;
  }
  err = cudaMemsetAsync(L->status, 0, sizeof(unsigned), L->stream);
  if (err == cudaSuccess)
    err = cudaMemsetAsync(L->ghost, 0, kGhostBlocks * kGhostStride * L->real_elem, L->stream);
  if (err == cudaSuccess)
    err = cudaMemsetAsync(L->wrho, 0,
                          (2 * (size_t)grid->nx * grid->nz + 2 * (size_t)grid->ny * grid->nz) * L->real_elem,
                          L->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(L->stream);
  if (err != cudaSuccess) {
    free_all(L);
    delete L;
    return cuda_fail(err, "rpk_create");
  }
  *out = L;
  return RPK_OK;
}

void rpk_destroy(rpk_lattice* L) {
  if (!L) return;
  cudaStreamSynchronize(L->stream);
  free_all(L);
  delete L;
}

rpk_status rpk_set_relax(rpk_lattice* L, const rpk_relax* r) {
  if (!L) return fail(RPK_ERR_ARG, "lattice is NULL");
  rpk_status st = validate_relax(r);
  if (st != RPK_OK) return st;
  L->relax = *r;
  L->relax_ok = true;
  if (r->nsub > 0) L->nsub = r->nsub;
  if (L->res_ok || L->walls || L->xwalls) {
    // the boundary tables hold e and kappa_R, which depend on the parameters
    RPK_CUDA(cudaSetDevice(L->device));
    return with_ops(L->grid.precision, [&](auto ops) { return decltype(ops)::ghosts(L); });
  }
  return RPK_OK;
}

rpk_status rpk_set_gas(rpk_lattice* L, double gamma, double eta, double eta_B, double kappa,
                       double b) {
  if (!L) return fail(RPK_ERR_ARG, "lattice is NULL");
  rpk_relax r;
  rpk_status st = rpk_map_gas(gamma, eta, eta_B, kappa, b, 1.0, &r);
  if (st != RPK_OK) return st;
  return rpk_set_relax(L, &r);
}

rpk_status rpk_set_reservoirs(rpk_lattice* L, const double* s) {
  if (!L || !s) return fail(RPK_ERR_ARG, "lattice or states is NULL");
  if (L->grid.bc_x != RPK_BC_RESERVOIR) return fail(RPK_ERR_STATE, "lattice is not RPK_BC_RESERVOIR");
  if (!L->relax_ok) return fail(RPK_ERR_STATE, "set the relaxation parameters first");
  for (int side = 0; side < 2; ++side) {
    const double* t = s + 6 * side;
    if (!(t[0] > 0.0) || !(t[4] > 0.0) || !(t[5] > 0.0))
      return fail(RPK_ERR_PARAM, "reservoir rho, theta_T, theta_R must be > 0");
    for (int k = 0; k < 6; ++k)
      if (!std::isfinite(t[k])) return fail(RPK_ERR_PARAM, "reservoir state not finite");
  }
  std::memcpy(L->res, s, sizeof(L->res));
  cudaError_t err = cudaSetDevice(L->device);
  if (err != cudaSuccess) return cuda_fail(err, "cudaSetDevice");
  rpk_status st = with_ops(L->grid.precision, [&](auto ops) { return decltype(ops)::ghosts(L); });
  if (st != RPK_OK) return st;
  L->res_ok = true;
  return RPK_OK;
}

rpk_status rpk_set_walls(rpk_lattice* L, const double* w) {
  if (!L) return fail(RPK_ERR_ARG, "lattice is NULL");
  if (!w) {
    L->walls = false;
    return RPK_OK;
  }
  if (L->grid.ny < 2) return fail(RPK_ERR_STATE, "walls need ny >= 2");
  if (L->grid.bc_x != RPK_BC_PERIODIC) return fail(RPK_ERR_STATE, "walls need a periodic x boundary");
  if (!L->relax_ok) return fail(RPK_ERR_STATE, "set the relaxation parameters first");
  for (int k = 0; k < 8; ++k)
    if (!std::isfinite(w[k])) return fail(RPK_ERR_PARAM, "wall state not finite");
  if (w[1] != 0.0 || w[5] != 0.0) return fail(RPK_ERR_PARAM, "walls slide tangentially: uy must be 0");
  if (!(w[3] > 0.0) || !(w[7] > 0.0)) return fail(RPK_ERR_PARAM, "wall temperatures must be > 0");
  std::memcpy(L->wall, w, sizeof(L->wall));
  L->walls = true;
  RPK_CUDA(cudaSetDevice(L->device));
  return with_ops(L->grid.precision, [&](auto ops) { return decltype(ops)::ghosts(L); });
}

rpk_status rpk_set_x_walls(rpk_lattice* L, const double* w) {
  if (!L) return fail(RPK_ERR_ARG, "lattice is NULL");
  if (!w) {
    L->xwalls = false;
    return RPK_OK;
  }
  if (L->grid.nx < 2) return fail(RPK_ERR_STATE, "x walls need nx >= 2");
  if (L->grid.bc_x != RPK_BC_PERIODIC) return fail(RPK_ERR_STATE, "x walls replace the x reservoirs: use bc_x = periodic");
  if (!L->relax_ok) return fail(RPK_ERR_STATE, "set the relaxation parameters first");
  for (int k = 0; k < 8; ++k)
    if (!std::isfinite(w[k])) return fail(RPK_ERR_PARAM, "wall state not finite");
  if (w[0] != 0.0 || w[4] != 0.0) return fail(RPK_ERR_PARAM, "walls slide tangentially: ux must be 0");
  if (!(w[3] > 0.0) || !(w[7] > 0.0)) return fail(RPK_ERR_PARAM, "wall temperatures must be > 0");
  std::memcpy(L->xwall, w, sizeof(L->xwall));
  L->xwalls = true;
  RPK_CUDA(cudaSetDevice(L->device));
  return with_ops(L->grid.precision, [&](auto ops) { return decltype(ops)::ghosts(L); });
}

rpk_status rpk_set_rot_mode(rpk_lattice* L, int mode) {
  if (!L) return fail(RPK_ERR_ARG, "lattice is NULL");
  if (mode != 0 && mode != 1) return fail(RPK_ERR_ARG, "mode must be 0 (conservative) or 1 (paper)");
  if (mode == L->rot_mode) return RPK_OK;
  L->rot_mode = mode;
  L->init_ok = false;  // the stored rotational state changes meaning: initialise again
  if (L->res_ok || L->walls || L->xwalls) {
    cudaError_t err = cudaSetDevice(L->device);
    if (err != cudaSuccess) return cuda_fail(err, "cudaSetDevice");
    return with_ops(L->grid.precision, [&](auto ops) { return decltype(ops)::ghosts(L); });
  }
  return RPK_OK;
}

static rpk_status ensure_stage(rpk_lattice* L) {
  if (L->stage) return RPK_OK;
  const size_t bytes = sizeof(double) * 7 * (size_t)L->npts;
  cudaError_t err = cudaMalloc(&L->stage, bytes);
  if (err != cudaSuccess) {
    L->stage = nullptr;
    cudaGetLastError();
    return fail(RPK_ERR_OOM, "staging allocation failed");
  }
  L->bytes_held += bytes;
  return RPK_OK;
}

// Device address under which the current device reads or writes host memory
// p in place: pinned (page-locked or registered) memory through its mapped
// device pointer, at the host link's full rate (NVLink-C2C on Grace
// systems). Pageable memory is not used in place even where the device could
// reach it: first-touch address translation made a kernel reading freshly
// allocated pageable arrays run at ~25 GB/s, slower than a staging copy.
static bool host_view(const rpk_lattice* L, const void* p, void** out) {
  (void)L;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) {
    *out = a.devicePointer;
    return true;
  }
  return false;
}

rpk_status rpk_init_fields(rpk_lattice* L, const double* rho, const double* u,
                           const double* T, const double* R, int on_device) {
  if (!L || !rho || !u || !T || !R) return fail(RPK_ERR_ARG, "NULL argument");
  if (!L->relax_ok) return fail(RPK_ERR_STATE, "set the relaxation parameters first");
  if (L->grid.bc_x == RPK_BC_RESERVOIR && !L->res_ok)
    return fail(RPK_ERR_STATE, "set the reservoirs first");
  RPK_CUDA(cudaSetDevice(L->device));
  const int64_t n = L->npts;
  const double *drho = rho, *du = u, *dT = T, *dR = R;
  if (!on_device) {
    // host fields: read in place by the initialisation kernel where the device
    // can reach them, otherwise one copy per field into the staging buffer
    void* v[4];
    if (host_view(L, rho, &v[0]) && host_view(L, u, &v[1]) && host_view(L, T, &v[2]) &&
        host_view(L, R, &v[3])) {
      drho = static_cast<const double*>(v[0]);
      du = static_cast<const double*>(v[1]);
      dT = static_cast<const double*>(v[2]);
      dR = static_cast<const double*>(v[3]);
    } else {
      rpk_status st = ensure_stage(L);
      if (st != RPK_OK) return st;
      double* s = L->stage;
      RPK_CUDA(cudaMemcpyAsync(s, rho, n * sizeof(double), cudaMemcpyHostToDevice, L->stream));
      RPK_CUDA(cudaMemcpyAsync(s + n, u, 3 * n * sizeof(double), cudaMemcpyHostToDevice, L->stream));
      RPK_CUDA(cudaMemcpyAsync(s + 4 * n, T, n * sizeof(double), cudaMemcpyHostToDevice, L->stream));
      RPK_CUDA(cudaMemcpyAsync(s + 5 * n, R, n * sizeof(double), cudaMemcpyHostToDevice, L->stream));
      drho = s;
      du = s + n;
      dT = s + 4 * n;
      dR = s + 5 * n;
    }
  }
  // one pass: the initial state, the check of the inputs and the largest theta
  L->init_ok = false;
  rpk_status st = with_ops(L->grid.precision,
                           [&](auto ops) { return decltype(ops)::init(L, drho, du, dT, dR); });
  if (st != RPK_OK) return st;
  unsigned long long check[2] = {0, 0};
  RPK_CUDA(cudaMemcpyAsync(check, L->diag_out, sizeof(check), cudaMemcpyDeviceToHost, L->stream));
  RPK_CUDA(cudaStreamSynchronize(L->stream));
  if (check[1] != 0)
    return fail(RPK_ERR_PARAM, "fields need finite rho > 0, theta_T > 0, theta_R > 0 and finite u");
  double tmax;
  std::memcpy(&tmax, &check[0], sizeof(double));
  tmax /= 3.0 + L->relax.delta;
  if (!(tmax > 0.0) || !std::isfinite(tmax)) return fail(RPK_ERR_PARAM, "fields need theta > 0");
  // FTCS sub-steps from the largest initial theta when nsub = 0
  if (L->relax.nsub == 0) {
    if (L->walls || L->xwalls) {
      // a point next to a wall has one face of coefficient 4 kappa_R (distance
      // 1/4) per wall axis
      if (L->walls) tmax = std::max(tmax, std::max(L->wall[3], L->wall[7]));
      if (L->xwalls) tmax = std::max(tmax, std::max(L->xwall[3], L->xwall[7]));
      L->nsub = nsub_for_diagonal(&L->relax, tmax,
                                  2.0 * active_dims(L->grid) + 3.0 * ((int)L->walls + (int)L->xwalls));
    } else {
      L->nsub = rpk_auto_nsub(&L->relax, tmax, active_dims(L->grid));
    }
  } else {
    L->nsub = L->relax.nsub;
  }
  RPK_CUDA(cudaMemsetAsync(L->status, 0, sizeof(unsigned), L->stream));
  RPK_CUDA(cudaStreamSynchronize(L->stream));
  L->streamed = true;
  L->steps = 0;
  L->init_ok = true;
  return RPK_OK;
}

rpk_status rpk_step(rpk_lattice* L, int64_t n) {
  if (!L) return fail(RPK_ERR_ARG, "lattice is NULL");
  if (n < 0) return fail(RPK_ERR_ARG, "n must be >= 0");
  if (!L->init_ok) return fail(RPK_ERR_STATE, "initialise the fields first");
  if (n == 0) return RPK_OK;
  RPK_CUDA(cudaSetDevice(L->device));
  return with_ops(L->grid.precision, [&](auto ops) { return decltype(ops)::step(L, n); });
}

static rpk_status read_status(rpk_lattice* L, unsigned* flags) {
  RPK_CUDA(cudaMemcpyAsync(flags, L->status, sizeof(unsigned), cudaMemcpyDeviceToHost, L->stream));
  RPK_CUDA(cudaStreamSynchronize(L->stream));
  return RPK_OK;
}

rpk_status rpk_read_moments(rpk_lattice* L, double* rho, double* u, double* T, double* R,
                            double* E, int on_device) {
  if (!L) return fail(RPK_ERR_ARG, "lattice is NULL");
  if (!L->init_ok) return fail(RPK_ERR_STATE, "initialise the fields first");
  RPK_CUDA(cudaSetDevice(L->device));
  const int64_t n = L->npts;
  double *o_rho = rho, *o_u = u, *o_T = T, *o_R = R, *o_E = E;
  bool staged = false;
  if (!on_device) {
    // host outputs: written in place by the moments kernel where the device
    // can reach them, otherwise through the staging buffer
    double* outs[5] = {rho, u, T, R, E};
    double* views[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool direct = true;
    for (int k = 0; k < 5 && direct; ++k) {
      void* v = nullptr;
      if (outs[k]) {
        direct = host_view(L, outs[k], &v);
        views[k] = static_cast<double*>(v);
      }
    }
    if (direct) {
      o_rho = views[0], o_u = views[1], o_T = views[2], o_R = views[3], o_E = views[4];
    } else {
      rpk_status st = ensure_stage(L);
      if (st != RPK_OK) return st;
      double* s = L->stage;
      o_rho = rho ? s : nullptr;
      o_u = u ? s + n : nullptr;
      o_T = T ? s + 4 * n : nullptr;
      o_R = R ? s + 5 * n : nullptr;
      o_E = E ? s + 6 * n : nullptr;
      staged = true;
    }
  }
  rpk_status st = with_ops(L->grid.precision, [&](auto ops) {
    return decltype(ops)::moments(L, o_rho, o_u, o_T, o_R, o_E);
  });
  if (st != RPK_OK) return st;
  if (staged) {
    const size_t b = n * sizeof(double);
    if (rho) RPK_CUDA(cudaMemcpyAsync(rho, o_rho, b, cudaMemcpyDeviceToHost, L->stream));
    if (u) RPK_CUDA(cudaMemcpyAsync(u, o_u, 3 * b, cudaMemcpyDeviceToHost, L->stream));
    if (T) RPK_CUDA(cudaMemcpyAsync(T, o_T, b, cudaMemcpyDeviceToHost, L->stream));
    if (R) RPK_CUDA(cudaMemcpyAsync(R, o_R, b, cudaMemcpyDeviceToHost, L->stream));
    if (E) RPK_CUDA(cudaMemcpyAsync(E, o_E, b, cudaMemcpyDeviceToHost, L->stream));
  }
  unsigned flags = 0;
  st = read_status(L, &flags);
  if (st != RPK_OK) return st;
  if (flags) return fail(RPK_ERR_NUMERIC, "device flagged a non-finite or non-positive moment");
  return RPK_OK;
}

rpk_status rpk_diagnostics(rpk_lattice* L, rpk_diag* out) {
  if (!L || !out) return fail(RPK_ERR_ARG, "NULL argument");
  if (!L->init_ok) return fail(RPK_ERR_STATE, "initialise the fields first");
  RPK_CUDA(cudaSetDevice(L->device));
  double v[kDiagVals];
  rpk_status st = with_ops(L->grid.precision, [&](auto ops) { return decltype(ops)::diag(L, v); });
  if (st != RPK_OK) return st;
  unsigned flags = 0;
  st = read_status(L, &flags);
  if (st != RPK_OK) return st;
  out->mass = v[0];
  out->mom[0] = v[1];
  out->mom[1] = v[2];
  out->mom[2] = v[3];
  out->energy = v[4];
  out->H1 = v[5];
  out->min_g = v[6];
  out->status = flags;
  out->pad = 0;
  out->steps = L->steps;
  if (flags) return fail(RPK_ERR_NUMERIC, "device flagged a non-finite or non-positive moment");
  return RPK_OK;
}

// ---- checkpoints -----------------------------------------------------------

namespace {
struct CkptHeader {
  char magic[8];
  int32_t abi;
  int32_t nx, ny, nz, precision, bc_x;
  int32_t nsub, streamed, res_ok;
  int64_t steps;
  rpk_relax relax;
  double res[12];
  int32_t rot_mode, walls;
  double wall[8];
  int32_t xwalls, pad;
  double xwall[8];
};
}  // namespace

static rpk_status copy_out(rpk_lattice* L, FILE* f, const void* dev, size_t bytes) {
  std::vector<char> buf(bytes);
  RPK_CUDA(cudaMemcpyAsync(buf.data(), dev, bytes, cudaMemcpyDeviceToHost, L->stream));
  RPK_CUDA(cudaStreamSynchronize(L->stream));
  if (fwrite(buf.data(), 1, bytes, f) != bytes) return fail(RPK_ERR_IO, "checkpoint write failed");
  return RPK_OK;
}

static rpk_status copy_in(rpk_lattice* L, FILE* f, void* dev, size_t bytes) {
  std::vector<char> buf(bytes);
  if (fread(buf.data(), 1, bytes, f) != bytes) return fail(RPK_ERR_IO, "checkpoint truncated");
  RPK_CUDA(cudaMemcpyAsync(dev, buf.data(), bytes, cudaMemcpyHostToDevice, L->stream));
  RPK_CUDA(cudaStreamSynchronize(L->stream));
  return RPK_OK;
}

rpk_status rpk_save(rpk_lattice* L, const char* path) {
  if (!L || !path) return fail(RPK_ERR_ARG, "NULL argument");
  if (!L->init_ok) return fail(RPK_ERR_STATE, "nothing to save");
  RPK_CUDA(cudaSetDevice(L->device));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(RPK_ERR_IO, std::string("cannot open ") + path);
  CkptHeader h{};
  std::memcpy(h.magic, "RPKCKPT4", 8);
  h.rot_mode = L->rot_mode;
  h.walls = L->walls;
  std::memcpy(h.wall, L->wall, sizeof(h.wall));
  h.xwalls = L->xwalls;
  std::memcpy(h.xwall, L->xwall, sizeof(h.xwall));
  h.abi = RPK_ABI_VERSION;
  h.nx = L->grid.nx; h.ny = L->grid.ny; h.nz = L->grid.nz;
  h.precision = L->grid.precision; h.bc_x = L->grid.bc_x;
  h.nsub = L->nsub; h.streamed = L->streamed; h.res_ok = L->res_ok;
  h.steps = L->steps;
  h.relax = L->relax;
  std::memcpy(h.res, L->res, sizeof(h.res));
  rpk_status st = RPK_OK;
  if (fwrite(&h, sizeof(h), 1, f) != 1) st = fail(RPK_ERR_IO, "checkpoint write failed");
  const size_t popb = (size_t)kQ * L->npts * L->store_elem, fb = (size_t)L->npts * L->real_elem;
  // u ring stored as (u(t-1), u(t)) in that order relative to the step count
  if (st == RPK_OK) st = copy_out(L, f, L->pop[L->cur], popb);
  if (st == RPK_OK) st = copy_out(L, f, L->e, fb);
  if (st == RPK_OK) st = copy_out(L, f, L->u[0], 3 * fb);
  if (st == RPK_OK) st = copy_out(L, f, L->u[1], 3 * fb);
  if (st == RPK_OK) st = copy_out(L, f, L->status, sizeof(unsigned));
  if (fclose(f) != 0 && st == RPK_OK) st = fail(RPK_ERR_IO, "checkpoint close failed");
  return st;
}

rpk_status rpk_load(rpk_lattice* L, const char* path) {
  if (!L || !path) return fail(RPK_ERR_ARG, "NULL argument");
  RPK_CUDA(cudaSetDevice(L->device));
  FILE* f = fopen(path, "rb");
  if (!f) return fail(RPK_ERR_IO, std::string("cannot open ") + path);
  CkptHeader h{};
  rpk_status st = RPK_OK;
  if (fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, "RPKCKPT4", 8) != 0)
    st = fail(RPK_ERR_IO, "not a checkpoint");
  else if ((h.walls && (h.bc_x != RPK_BC_PERIODIC || h.ny < 2)) ||
           (h.xwalls && (h.bc_x != RPK_BC_PERIODIC || h.nx < 2)))
    st = fail(RPK_ERR_IO, "inconsistent checkpoint");
  else if (h.rot_mode != L->rot_mode)
    st = fail(RPK_ERR_ARG, "checkpoint rotational mode differs from the lattice (rpk_set_rot_mode)");
  else if (h.nx != L->grid.nx || h.ny != L->grid.ny || h.nz != L->grid.nz ||
           h.precision != L->grid.precision || h.bc_x != L->grid.bc_x)
    st = fail(RPK_ERR_ARG, "checkpoint grid differs from the lattice");
  if (st == RPK_OK) st = validate_relax(&h.relax);
  const size_t popb = (size_t)kQ * L->npts * L->store_elem, fb = (size_t)L->npts * L->real_elem;
  if (st == RPK_OK) st = copy_in(L, f, L->pop[0], popb);
  if (st == RPK_OK) st = copy_in(L, f, L->e, fb);
  if (st == RPK_OK) st = copy_in(L, f, L->u[0], 3 * fb);
  if (st == RPK_OK) st = copy_in(L, f, L->u[1], 3 * fb);
  if (st == RPK_OK) st = copy_in(L, f, L->status, sizeof(unsigned));
  fclose(f);
  if (st != RPK_OK) {
    L->init_ok = false;
    return st;
  }
  L->relax = h.relax;
  L->relax_ok = true;
  L->nsub = h.nsub;
  L->streamed = h.streamed != 0;
  L->steps = h.steps;
  L->cur = 0;
  std::memcpy(L->res, h.res, sizeof(L->res));
  L->res_ok = h.res_ok != 0;
  L->walls = h.walls != 0;
  std::memcpy(L->wall, h.wall, sizeof(L->wall));
  L->xwalls = h.xwalls != 0;
  std::memcpy(L->xwall, h.xwall, sizeof(L->xwall));
  if (L->res_ok || L->walls || L->xwalls) {
    st = with_ops(L->grid.precision, [&](auto ops) { return decltype(ops)::ghosts(L); });
    if (st != RPK_OK) return st;
  }
  L->init_ok = true;
  return RPK_OK;
}

rpk_status rpk_timing(rpk_lattice* L, int enable) {
  if (!L) return fail(RPK_ERR_ARG, "lattice is NULL");
  L->timing = enable != 0;
  L->ev_used = 0;
  return RPK_OK;
}

rpk_status rpk_timing_read(rpk_lattice* L, double* ms, int64_t* launches) {
  if (!L || !ms || !launches) return fail(RPK_ERR_ARG, "NULL argument");
  RPK_CUDA(cudaSetDevice(L->device));
  RPK_CUDA(cudaStreamSynchronize(L->stream));
  for (int c = 0; c < RPK_KC_COUNT; ++c) {
    ms[c] = 0.0;
    launches[c] = 0;
  }
  for (size_t i = 0; i < L->ev_used; ++i) {
    float t = 0.f;
    RPK_CUDA(cudaEventElapsedTime(&t, L->events[2 * i], L->events[2 * i + 1]));
    ms[L->ev_class[i]] += t;
    launches[L->ev_class[i]] += L->ev_kernels[i];
  }
  return RPK_OK;
}

rpk_status rpk_get_info(rpk_lattice* L, int64_t out[4]) {
  if (!L || !out) return fail(RPK_ERR_ARG, "NULL argument");
  out[0] = L->nsub;
  out[1] = L->steps;
  out[2] = L->npts;
  out[3] = (int64_t)L->bytes_held;
  return RPK_OK;
}

}  // extern "C"
