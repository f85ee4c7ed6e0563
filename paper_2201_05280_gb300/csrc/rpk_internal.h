// Internal declarations shared by the C-ABI layer (rpk_api.cu) and the
// per-precision kernel launchers (rpk_ops_*.cu). Not part of the public API.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rpk.h"

struct rpk_lattice {
  rpk_grid grid;
  int device = 0;
  int sms = 1;           // streaming multiprocessors of the device
  cudaStream_t stream = nullptr;
  rpk_relax relax{};
  bool relax_ok = false;
  bool init_ok = false;
  bool res_ok = false;
  double res[12] = {0};
  int nsub = 1;          // FTCS sub-steps in use
  int rot_mode = 0;      // 0 conservative rotational transport, 1 the paper's theta_R solver
  int64_t n3 = 0, npts = 0;
  size_t store_elem = 0;  // bytes per stored population
  size_t real_elem = 0;   // bytes per field value
  void* pop[2] = {nullptr, nullptr};
  int cur = 0;            // buffer holding the current state
  bool streamed = true;   // current state is post-stream (after init/load)
  void* e = nullptr;      // auxiliary rotational energy (deviation), state
  void* e_star = nullptr; // after the exchange
  void* e_a = nullptr;    // transport scratch
  void* e_b = nullptr;    // transport scratch
  void* vbuf = nullptr;   // advecting velocity of the step (3 planes)
  void* thbuf = nullptr;  // theta_R - theta0 after advection
  void* drho = nullptr;
  void* kap = nullptr;
  void* u[2] = {nullptr, nullptr};  // ring: u(t) and u(t-1), 3 planes each
  void* ghost = nullptr;            // reservoir and wall table (Real, 4 x 48)
  bool walls = false;               // diffuse walls normal to y (rpk_set_walls)
  double wall[8] = {0};             // ux, uy, uz, theta of the low and the high y wall
  bool xwalls = false;              // diffuse walls normal to x (rpk_set_x_walls)
  double xwall[8] = {0};            // ux, uy, uz, theta of the low and the high x wall
  void* wrho = nullptr;             // rho_w - 1 per wall column (Real, 2 nx nz + 2 ny nz)
  unsigned* status = nullptr;
  double* diag_partial = nullptr;
  double* diag_out = nullptr;
  double* stage = nullptr;          // 7 x npts doubles for host I/O, lazy
  int64_t steps = 0;
  size_t bytes_held = 0;
  // kernel timing: event pairs recorded around each kernel class
  bool timing = false;
  std::vector<cudaEvent_t> events;
  std::vector<int> ev_class;   // class of each recorded pair
  std::vector<int> ev_kernels; // kernel launches inside each pair
  size_t ev_used = 0;          // pairs recorded since the last start
};

namespace rpk {
// Record the start / end of a timed kernel class (no-ops unless timing is on).
cudaError_t timing_begin(rpk_lattice* L);
cudaError_t timing_end(rpk_lattice* L, int cls, int kernels);
}  // namespace rpk

namespace rpk {

// Thread-local error message of the last failed call.
void set_error(const std::string& msg);
rpk_status fail(rpk_status st, const std::string& msg);
rpk_status cuda_fail(cudaError_t err, const char* what);
// Parameter checks of rpk_set_relax.
rpk_status validate_relax(const rpk_relax* r);

#define RPK_CUDA(call)                                      \
  do {                                                      \
    cudaError_t err_ = (call);                              \
    if (err_ != cudaSuccess) return rpk::cuda_fail(err_, #call); \
  } while (0)

// Per-precision entry points (defined in rpk_ops.cuh, instantiated per TU).
template <typename Store, typename Real>
struct Ops {
  static rpk_status step(rpk_lattice* L, int64_t n);
  static rpk_status init(rpk_lattice* L, const double* rho, const double* u, const double* T,
                         const double* R);
  static rpk_status moments(rpk_lattice* L, double* rho, double* u, double* T, double* R,
                            double* E);
  static rpk_status diag(rpk_lattice* L, double out[8]);
  static rpk_status ghosts(rpk_lattice* L);
};

}  // namespace rpk
