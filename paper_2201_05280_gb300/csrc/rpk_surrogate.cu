// Surrogate rollout of batched quasi-1-D tubes: packing of network inputs and
// training targets, the conservative update from the network's increments, and
// the rollout engine that hands tubes back to the batched LBM (spot checks,
// drift and validity checks, final fallback run). The paper has no learned
// component; the LBM it drives is the paper's method (rpk_batch_*).
//
// Moment blocks: per tube [4][2 nx] floats (rho, u_x, theta_T, E_R). Point
// (s, x) of a tube sits at fine position 2x + s (half the sublattice spacing),
// which is the sequence order the network sees.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "rpk_internal.h"

namespace {

constexpr int kCin = 11, kCout = 4;

struct Norm {
  float shift[4], scale[4], out_scale[4], dscale[4];
  float noise[4];  // training-input perturbation: uniform, standard deviation noise[k]
  unsigned long long seed;
  int pad, project;
};

Norm make_norm(const rpk_sur_config* c) {
  Norm n;
  for (int k = 0; k < 4; ++k) {
    n.shift[k] = c->in_shift[k];
    n.scale[k] = c->in_scale[k];
    n.out_scale[k] = c->out_scale[k];
    n.dscale[k] = c->in_dscale[k];
  }
  n.pad = c->pad;
  n.project = c->project;
  for (int k = 0; k < 4; ++k) n.noise[k] = 0.f;
  n.seed = 0;
  return n;
}

// Conserved densities of (rho, u_x, theta_T, E_R).
__device__ __forceinline__ void conserved(const double v[4], double U[4]) {
  U[0] = v[0];
  U[1] = v[0] * v[1];
  U[2] = 0.5 * v[0] * v[1] * v[1] + 1.5 * v[0] * v[2] + v[3];
  U[3] = v[3];
}

__device__ __forceinline__ void load_point(const float* blk, int np, int pt, double v[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = (double)blk[(int64_t)k * np + pt];
}

// Output number n + 1 of the SplitMix64 generator seeded with `seed` (Steele,
// Lea & Flood, OOPSLA 2014): the state after n + 1 increments of the golden
// gamma, through the generator's output mix.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Fine position p of a tube -> its point index s nx + x.
__device__ __forceinline__ int point_of(int nx, int p) { return (p & 1) * nx + (p >> 1); }

__global__ void k_pack(const float* __restrict__ store, const float* __restrict__ prev_store,
                       const rpk_sur_seq* __restrict__ seqs, Norm N, int margin,
                       float* __restrict__ x, float* __restrict__ target, float* __restrict__ mask) {
  const rpk_sur_seq& S = seqs[blockIdx.y];
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= S.len) return;
  const int np = 2 * S.nx;
  const int p = S.crop + l - N.pad;
  const bool inside = p >= 0 && p < np;
  double v[4], q[4];
  if (inside) {
    load_point(store + S.src, np, point_of(S.nx, p), v);
    // perturbed source state (training only): v_k + noise_k sqrt(3) (2 u - 1), u uniform
    // in [0, 1) from draw ((sequence << 32 | l) * 4 + k)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (N.noise[k] != 0.f) {
        const uint64_t h = splitmix64(N.seed, ((((uint64_t)blockIdx.y) << 32) | (uint64_t)l) * 4 + k);
        const double u = (double)(h >> 11) * 0x1.0p-53;
        v[k] += (double)N.noise[k] * 1.7320508075688772 * (2.0 * u - 1.0);
      }
    if (S.prev >= 0)
      load_point(prev_store + S.prev, np, point_of(S.nx, p), q);
    else
#pragma unroll
      for (int k = 0; k < 4; ++k) q[k] = v[k];
  } else {
    const int side = p < 0 ? 0 : 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = v[k] = (double)S.res[side][k];
  }
  float* xo = x + (S.out + l) * kCin;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    xo[k] = ((float)v[k] - N.shift[k]) / N.scale[k];
    xo[4 + k] = ((float)v[k] - (float)q[k]) / N.dscale[k];
  }
  xo[8] = S.cond[0];
  xo[9] = S.cond[1];
  xo[10] = inside ? 1.f : 0.f;
  if (S.tgt < 0 || !target) return;
  const bool use = inside && l >= margin && l < S.len - margin;
  float* to = target + (S.out + l) * kCout;
  if (use) {
    double w[4], U0[4], U1[4];
    load_point(store + S.tgt, np, point_of(S.nx, p), w);
    conserved(v, U0);
    conserved(w, U1);
#pragma unroll
    for (int k = 0; k < 4; ++k) to[k] = (float)((U1[k] - U0[k]) / (double)N.out_scale[k]);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) to[k] = 0.f;
  }
  if (mask) mask[S.out + l] = use ? 1.f : 0.f;
}

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
  // red: NV x 32 doubles; blockDim.x a multiple of 32, <= 1024
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i * 32 + warp] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[i * 32 + w];  // fixed order: deterministic
    v[i] = t;
  }
}

// Increments of U at tube position p (scaled network outputs).
__device__ __forceinline__ void increments(const float* __restrict__ y, const rpk_sur_seq& S,
                                           const Norm& N, int p, double d[4]) {
  const float* yo = y + (S.out + N.pad + p - S.crop) * kCout;
#pragma unroll
  for (int k = 0; k < 4; ++k) d[k] = (double)N.out_scale[k] * (double)yo[k];
}

// One block per tube: projection sums, then the update, validity and totals.
__global__ void k_apply(const float* __restrict__ state, const float* __restrict__ y,
                        const rpk_sur_seq* __restrict__ seqs, Norm N, float* __restrict__ next,
                        int* __restrict__ flags, double* __restrict__ totals) {
  __shared__ double red[4 * 32];
  const rpk_sur_seq& S = seqs[blockIdx.x];
  const int np = 2 * S.nx;
  const float* in = state + S.src;
  float* out = next + S.src;
  // sums and absolute sums of the mass and energy increments
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  if (N.project) {
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
      double d[4];
      increments(y, S, N, p, d);
      a[0] += d[0];
      a[1] += fabs(d[0]);
      a[2] += d[2];
      a[3] += fabs(d[2]);
    }
    block_sum<4>(a, red);
  }
  const double c0 = (N.project && a[1] > 0.0) ? a[0] / a[1] : 0.0;
  const double c2 = (N.project && a[3] > 0.0) ? a[2] / a[3] : 0.0;
  double t[3] = {0.0, 0.0, 0.0};  // mass, energy, invalid count
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const int pt = point_of(S.nx, p);
    double v[4], U[4], d[4];
    load_point(in, np, pt, v);
    conserved(v, U);
    increments(y, S, N, p, d);
    d[0] -= fabs(d[0]) * c0;
    d[2] -= fabs(d[2]) * c2;
#pragma unroll
    for (int k = 0; k < 4; ++k) U[k] += d[k];
    const double rho = U[0], ux = U[1] / rho, er = U[3];
    const double th = (U[2] - 0.5 * U[1] * ux - er) / (1.5 * rho);
    const bool ok = rho > 0.0 && th > 0.0 && er > 0.0 && isfinite(rho) && isfinite(ux) &&
                    isfinite(th) && isfinite(er);
    out[pt] = (float)rho;
    out[np + pt] = (float)ux;
    out[2 * np + pt] = (float)th;
    out[3 * np + pt] = (float)er;
    t[0] += rho;
    t[1] += U[2];
    t[2] += ok ? 0.0 : 1.0;
  }
  block_sum<3>(t, red);
  if (threadIdx.x == 0) {
    flags[blockIdx.x] = t[2] > 0.0 ? 1 : 0;
    totals[2 * blockIdx.x] = t[0];
    totals[2 * blockIdx.x + 1] = t[1];
  }
}

// Per tube: sum |rho_a - rho_b| and sum |rho_b| (FP64).
__global__ void k_l1(const float* __restrict__ a, const float* __restrict__ b,
                     const rpk_sur_seq* __restrict__ seqs, double* __restrict__ out) {
  __shared__ double red[2 * 32];
  const rpk_sur_seq& S = seqs[blockIdx.x];
  const int np = 2 * S.nx;
  double t[2] = {0.0, 0.0};
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const double x = a[S.src + p], r = b[S.src + p];
    t[0] += fabs(x - r);
    t[1] += fabs(r);
  }
  block_sum<2>(t, red);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = t[0];
    out[2 * blockIdx.x + 1] = t[1];
  }
}

// Mass and energy totals of moment blocks, per tube.
__global__ void k_totals(const float* __restrict__ state, const rpk_sur_seq* __restrict__ seqs,
                         double* __restrict__ totals) {
  __shared__ double red[2 * 32];
  const rpk_sur_seq& S = seqs[blockIdx.x];
  const int np = 2 * S.nx;
  double t[2] = {0.0, 0.0};
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    double v[4], U[4];
    load_point(state + S.src, np, p, v);
    conserved(v, U);
    t[0] += U[0];
    t[1] += U[2];
  }
  block_sum<2>(t, red);
  if (threadIdx.x == 0) {
    totals[2 * blockIdx.x] = t[0];
    totals[2 * blockIdx.x + 1] = t[1];
  }
}

// flags[i] = 1 where a tube's moment block holds a non-positive rho, theta_T or
// E_R, or a non-finite value.
__global__ void k_valid(const float* __restrict__ state, const rpk_sur_seq* __restrict__ seqs,
                        int* __restrict__ flags) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const rpk_sur_seq& S = seqs[blockIdx.x];
  const int np = 2 * S.nx;
  const float* b = state + S.src;
  bool mine = false;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const float r = b[p], u = b[np + p], th = b[2 * np + p], er = b[3 * np + p];
    mine |= !(r > 0.f) || !(th > 0.f) || !(er > 0.f) || !isfinite(r) || !isfinite(u) ||
            !isfinite(th) || !isfinite(er);
  }
  if (mine) bad = 1;
  __syncthreads();
  if (threadIdx.x == 0) flags[blockIdx.x] = bad;
}

// Copy whole moment blocks src -> dst for the listed tubes.
__global__ void k_copy_blocks(const float* __restrict__ src, float* __restrict__ dst,
                              const rpk_sur_seq* __restrict__ seqs) {
  const rpk_sur_seq& S = seqs[blockIdx.x];
  const int64_t n = 8 * (int64_t)S.nx;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) dst[S.src + i] = src[S.src + i];
}

rpk_status check_config(const rpk_sur_config* c) {
  if (!c) return rpk::fail(RPK_ERR_ARG, "NULL configuration");
  if (c->jump < 1 || c->pad < 0 || c->pad % 4 || c->spot_every < 0)
    return rpk::fail(RPK_ERR_ARG, "jump >= 1, pad >= 0 a multiple of 4, spot_every >= 0");
  for (int k = 0; k < 4; ++k)
    if (!(c->in_scale[k] != 0.f) || !(c->out_scale[k] != 0.f) || !(c->in_dscale[k] != 0.f) ||
        !std::isfinite(c->in_scale[k]) || !std::isfinite(c->out_scale[k]) ||
        !std::isfinite(c->in_dscale[k]) || !std::isfinite(c->in_shift[k]))
      return rpk::fail(RPK_ERR_ARG, "scales must be finite and non-zero");
  return RPK_OK;
}

}  // namespace

struct rpk_rollout {
  rpk_net* net = nullptr;
  rpk_sur_config cfg{};
  int ntubes = 0, device = 0;
  cudaStream_t stream = nullptr;
  std::vector<rpk_tube> tubes;
  std::vector<float> cond;
  std::vector<int64_t> blk;  // float offset of each tube's moment block
  int64_t state_floats = 0, seq_points = 0;
  rpk_batch* batch = nullptr;
  float *next = nullptr, *lbm = nullptr, *init = nullptr, *prev = nullptr, *x = nullptr, *y = nullptr;
  std::vector<double> trace;  // per tube and window: spot-check L1 error (NaN: no check)
  int trace_windows = 0;
  rpk_sur_seq* seqs = nullptr;   // ntubes sequence descriptors (active tubes first)
  rpk_sur_seq* lists = nullptr;  // 2 x ntubes descriptors for block copies
  int* flags = nullptr;
  double* sums = nullptr;  // 2 x ntubes totals, 2 x ntubes L1 sums
  cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace {

rpk_status ro_alloc(void** p, size_t bytes) {
  cudaError_t err = cudaMalloc(p, bytes);
  if (err != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return rpk::fail(RPK_ERR_OOM, std::string("rollout allocation failed: ") + cudaGetErrorString(err));
  }
  return RPK_OK;
}

void free_rollout(rpk_rollout* R) {
  if (R->batch) rpk_batch_destroy(R->batch);
  void* p[] = {R->next, R->lbm, R->init, R->prev, R->x, R->y, R->seqs, R->lists, R->flags, R->sums};
  for (void* q : p)
    if (q) cudaFree(q);
  for (auto& e : R->ev)
    if (e) cudaEventDestroy(e);
}

int seq_len(const rpk_rollout* R, int tube) {
  const int n = 2 * R->tubes[tube].nx + 2 * R->cfg.pad;
  return (n + 3) / 4 * 4;
}

// The moment-block values (rho, u_x, theta_T, E_R = delta rho theta_R / 2,
// eq. thetadef's rotational energy) of a tube's low and high reservoir states.
void tube_reservoir_moments(const rpk_tube& t, float* out8) {
  for (int side = 0; side < 2; ++side) {
    const double* r = t.res + 6 * side;
    out8[4 * side + 0] = (float)r[0];
    out8[4 * side + 1] = (float)r[1];
    out8[4 * side + 2] = (float)r[4];
    out8[4 * side + 3] = (float)(0.5 * t.relax.delta * r[0] * r[5]);
  }
}

rpk_sur_seq make_seq(const rpk_rollout* R, int tube, int64_t out) {
  rpk_sur_seq s;
  std::memset(&s, 0, sizeof(s));
  const rpk_tube& t = R->tubes[tube];
  s.src = R->blk[tube];
  s.tgt = -1;
  s.prev = -1;
  s.out = out;
  s.nx = t.nx;
  s.len = seq_len(R, tube);
  s.crop = 0;
  tube_reservoir_moments(t, &s.res[0][0]);
  s.cond[0] = R->cond[2 * tube];
  s.cond[1] = R->cond[2 * tube + 1];
  return s;
}

// Copy the moment blocks of `ids` from src to dst.
rpk_status copy_blocks(rpk_rollout* R, const float* src, float* dst, const std::vector<int>& ids,
                       rpk_sur_seq* dev_list) {
  if (ids.empty()) return RPK_OK;
  std::vector<rpk_sur_seq> h(ids.size());
  for (size_t i = 0; i < ids.size(); ++i) h[i] = make_seq(R, ids[i], 0);
  RPK_CUDA(cudaMemcpyAsync(dev_list, h.data(), sizeof(rpk_sur_seq) * h.size(),
                           cudaMemcpyHostToDevice, R->stream));
  k_copy_blocks<<<(unsigned)ids.size(), 256, 0, R->stream>>>(src, dst, dev_list);
  RPK_CUDA(cudaGetLastError());
  RPK_CUDA(cudaStreamSynchronize(R->stream));  // h is released on return
  return RPK_OK;
}

// One LBM run of `steps` per tube from the moment blocks `from`; moments to R->lbm.
rpk_status lbm_run(rpk_rollout* R, const float* from, const std::vector<int>& steps) {
  rpk_status st = rpk_batch_set_steps(R->batch, steps.data());
  if (st == RPK_OK) st = rpk_batch_init_device(R->batch, from);
  if (st == RPK_OK) st = rpk_batch_run(R->batch);
  if (st == RPK_OK) st = rpk_batch_moments_device(R->batch, R->lbm);
  return st;
}

float elapsed(rpk_rollout* R) {
  float ms = 0.f;
  cudaEventSynchronize(R->ev[1]);
  cudaEventElapsedTime(&ms, R->ev[0], R->ev[1]);
  return ms;
}

}  // namespace

extern "C" {

rpk_status rpk_sur_reservoirs(const rpk_tube* tube, float* out) {
  if (!tube || !out) return rpk::fail(RPK_ERR_ARG, "NULL argument");
  tube_reservoir_moments(*tube, out);
  return RPK_OK;
}

rpk_status rpk_sur_pack(const rpk_sur_config* cfg, const float* store, const rpk_sur_seq* seqs,
                        int nseq, int maxlen, int margin, const float* noise, uint64_t seed,
                        float* x, float* target, float* mask, void* cuda_stream) {
  rpk_status st = check_config(cfg);
  if (st != RPK_OK) return st;
  if (!store || !seqs || !x) return rpk::fail(RPK_ERR_ARG, "NULL argument");
  if (nseq < 0 || maxlen < 0 || margin < 0 || nseq > 65535)
    return rpk::fail(RPK_ERR_ARG, "0 <= nseq <= 65535, maxlen >= 0, margin >= 0");
  if (nseq == 0 || maxlen == 0) return RPK_OK;
  Norm N = make_norm(cfg);
  if (noise)
    for (int k = 0; k < 4; ++k) {
      if (!(noise[k] >= 0.f) || !std::isfinite(noise[k])) return rpk::fail(RPK_ERR_ARG, "noise must be >= 0");
      N.noise[k] = noise[k];
    }
  N.seed = seed;
  const dim3 grid((unsigned)((maxlen + 255) / 256), (unsigned)nseq);
  k_pack<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(store, store, seqs, N, margin, x,
                                                                    target, mask);
  RPK_CUDA(cudaGetLastError());
  return RPK_OK;
}

rpk_status rpk_sur_apply(const rpk_sur_config* cfg, const float* state, const float* y,
                         const rpk_sur_seq* seqs, int nseq, float* next, int* flags,
                         double* totals, void* cuda_stream) {
  rpk_status st = check_config(cfg);
  if (st != RPK_OK) return st;
  if (!state || !y || !seqs || !next || !flags || !totals) return rpk::fail(RPK_ERR_ARG, "NULL argument");
  if (nseq < 0) return rpk::fail(RPK_ERR_ARG, "nseq < 0");
  if (nseq == 0) return RPK_OK;
  k_apply<<<(unsigned)nseq, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      state, y, seqs, make_norm(cfg), next, flags, totals);
  RPK_CUDA(cudaGetLastError());
  return RPK_OK;
}

rpk_status rpk_rollout_create(rpk_net* net, const rpk_sur_config* cfg, int ntubes,
                              const rpk_tube* tubes, const float* cond, void* cuda_stream,
                              rpk_rollout** out) {
  if (!out) return rpk::fail(RPK_ERR_ARG, "out is NULL");
  *out = nullptr;
  rpk_status st = check_config(cfg);
  if (st != RPK_OK) return st;
  if (!net || !tubes || !cond || ntubes < 1) return rpk::fail(RPK_ERR_ARG, "NULL argument or ntubes < 1");
  if (ntubes > 65535) return rpk::fail(RPK_ERR_ARG, "at most 65535 tubes");
  for (int i = 0; i < ntubes; ++i)
    if (tubes[i].relax.nsub < 1)
      return rpk::fail(RPK_ERR_ARG, "tube " + std::to_string(i) + ": relax.nsub must be > 0");
  rpk_rollout* R = new (std::nothrow) rpk_rollout();
  if (!R) return rpk::fail(RPK_ERR_OOM, "host allocation failed");
  R->net = net;
  R->cfg = *cfg;
  R->ntubes = ntubes;
  R->stream = static_cast<cudaStream_t>(cuda_stream);
  R->tubes.assign(tubes, tubes + ntubes);
  R->cond.assign(cond, cond + 2 * (size_t)ntubes);
  cudaGetDevice(&R->device);
  R->blk.resize(ntubes);
  for (int i = 0; i < ntubes; ++i) {
    R->blk[i] = R->state_floats;
    R->state_floats += 8 * (int64_t)tubes[i].nx;
    R->seq_points += seq_len(R, i);
  }
  st = rpk_batch_create(RPK_F32, ntubes, tubes, 1 << 30, cuda_stream, &R->batch);
  if (st == RPK_OK) st = rpk_batch_set_diffusion(R->batch, cfg->lbm_diffusion);
  if (st == RPK_OK && cfg->lbm_threads > 0)
    st = rpk_batch_set_config(R->batch, cfg->lbm_threads, std::max(1, cfg->lbm_ctas_per_sm));
  if (st == RPK_OK) st = ro_alloc((void**)&R->next, sizeof(float) * R->state_floats);
  if (st == RPK_OK) st = ro_alloc((void**)&R->lbm, sizeof(float) * R->state_floats);
  if (st == RPK_OK) st = ro_alloc((void**)&R->init, sizeof(float) * R->state_floats);
  if (st == RPK_OK) st = ro_alloc((void**)&R->prev, sizeof(float) * R->state_floats);
  if (st == RPK_OK) st = ro_alloc((void**)&R->x, sizeof(float) * kCin * R->seq_points);
  if (st == RPK_OK) st = ro_alloc((void**)&R->y, sizeof(float) * kCout * R->seq_points);
  if (st == RPK_OK) st = ro_alloc((void**)&R->seqs, sizeof(rpk_sur_seq) * ntubes);
  if (st == RPK_OK) st = ro_alloc((void**)&R->lists, sizeof(rpk_sur_seq) * 2 * ntubes);
  if (st == RPK_OK) st = ro_alloc((void**)&R->flags, sizeof(int) * ntubes);
  if (st == RPK_OK) st = ro_alloc((void**)&R->sums, sizeof(double) * 4 * ntubes);
  if (st == RPK_OK && (cudaEventCreate(&R->ev[0]) != cudaSuccess || cudaEventCreate(&R->ev[1]) != cudaSuccess))
    st = rpk::fail(RPK_ERR_CUDA, "event creation failed");
  if (st != RPK_OK) {
    free_rollout(R);
    delete R;
    return st;
  }
  *out = R;
  return RPK_OK;
}

void rpk_rollout_destroy(rpk_rollout* R) {
  if (!R) return;
  cudaStreamSynchronize(R->stream);
  free_rollout(R);
  delete R;
}

rpk_status rpk_rollout_run(rpk_rollout* R, float* state, int64_t* stats, double* est_out, double* ms) {
  if (!R || !state) return rpk::fail(RPK_ERR_ARG, "NULL argument");
  RPK_CUDA(cudaSetDevice(R->device));
  const int T = R->ntubes, jump = R->cfg.jump, C = R->cfg.spot_every;
  std::vector<int> J(T), fail_step(T, -1), windows(T, 0), checks(T, 0);
  std::vector<double> est(T, 0.0), M0(T), E0(T);
  double t_net = 0.0, t_spot = 0.0, t_fb = 0.0;
  int maxJ = 0;
  for (int i = 0; i < T; ++i) {
    J[i] = R->tubes[i].nsteps / jump;
    maxJ = std::max(maxJ, J[i]);
  }
  // reference totals
  {
    std::vector<rpk_sur_seq> h(T);
    for (int i = 0; i < T; ++i) h[i] = make_seq(R, i, 0);
    RPK_CUDA(cudaMemcpyAsync(R->seqs, h.data(), sizeof(rpk_sur_seq) * T, cudaMemcpyHostToDevice, R->stream));
    k_totals<<<T, 256, 0, R->stream>>>(state, R->seqs, R->sums);
    RPK_CUDA(cudaGetLastError());
    std::vector<double> tot(2 * T);
    RPK_CUDA(cudaMemcpyAsync(tot.data(), R->sums, sizeof(double) * 2 * T, cudaMemcpyDeviceToHost, R->stream));
    RPK_CUDA(cudaStreamSynchronize(R->stream));
    for (int i = 0; i < T; ++i) {
      M0[i] = tot[2 * i];
      E0[i] = tot[2 * i + 1];
    }
  }
  RPK_CUDA(cudaMemcpyAsync(R->init, state, sizeof(float) * R->state_floats, cudaMemcpyDeviceToDevice,
                           R->stream));
  R->trace.assign((size_t)T * std::max(maxJ, 1), std::nan(""));
  R->trace_windows = maxJ;
  const Norm N = make_norm(&R->cfg);
  std::vector<int> active, lens, steps(T);
  std::vector<char> has_prev(T, 0);
  std::vector<rpk_sur_seq> h;
  std::vector<int> flags(T);
  std::vector<double> sums(4 * T);
  for (int j = 0; j < maxJ; ++j) {
    active.clear();
    for (int i = 0; i < T; ++i)
      if (j < J[i] && fail_step[i] < 0) active.push_back(i);
    if (active.empty()) break;
    const int A = (int)active.size();
    h.resize(A);
    lens.resize(A);
    int64_t off = 0;
    for (int a = 0; a < A; ++a) {
      h[a] = make_seq(R, active[a], off);
      if (has_prev[active[a]]) h[a].prev = h[a].src;  // the same block of R->prev
      lens[a] = h[a].len;
      off += h[a].len;
    }
    const bool spot = C > 0 && j % C == 0;
    cudaEventRecord(R->ev[0], R->stream);
    RPK_CUDA(cudaMemcpyAsync(R->seqs, h.data(), sizeof(rpk_sur_seq) * A, cudaMemcpyHostToDevice, R->stream));
    int maxlen = *std::max_element(lens.begin(), lens.end());
    k_pack<<<dim3((maxlen + 255) / 256, A), 256, 0, R->stream>>>(state, R->prev, R->seqs, N, 0, R->x,
                                                                 nullptr, nullptr);
    RPK_CUDA(cudaGetLastError());
    // the network runs on its own stream: the packed inputs must be complete
    RPK_CUDA(cudaStreamSynchronize(R->stream));
    rpk_status st = rpk_net_forward_ragged(R->net, R->x, A, lens.data(), R->y);
    if (st != RPK_OK) return st;
    k_apply<<<A, 256, 0, R->stream>>>(state, R->y, R->seqs, N, R->next, R->flags, R->sums);
    RPK_CUDA(cudaGetLastError());
    cudaEventRecord(R->ev[1], R->stream);
    t_net += elapsed(R);
    if (spot) {
      for (int i = 0; i < T; ++i) steps[i] = 0;
      for (int i : active) steps[i] = jump;
      cudaEventRecord(R->ev[0], R->stream);
      st = lbm_run(R, state, steps);
      if (st != RPK_OK) return st;
      k_l1<<<A, 256, 0, R->stream>>>(R->next, R->lbm, R->seqs, R->sums + 2 * T);
      RPK_CUDA(cudaGetLastError());
      cudaEventRecord(R->ev[1], R->stream);
      t_spot += elapsed(R);
    }
    RPK_CUDA(cudaMemcpyAsync(flags.data(), R->flags, sizeof(int) * A, cudaMemcpyDeviceToHost, R->stream));
    RPK_CUDA(cudaMemcpyAsync(sums.data(), R->sums, sizeof(double) * 4 * T, cudaMemcpyDeviceToHost, R->stream));
    RPK_CUDA(cudaStreamSynchronize(R->stream));
    std::vector<int> from_next, from_lbm, from_init;
    const bool anchor = R->cfg.anchor != 0;
    for (int a = 0; a < A; ++a) {
      const int i = active[a];
      const double dm = std::fabs(sums[2 * a] - M0[i]) / std::fabs(M0[i]);
      const double de = std::fabs(sums[2 * a + 1] - E0[i]) / std::fabs(E0[i]);
      const bool valid = !flags[a] && dm <= R->cfg.drift_tol && de <= R->cfg.drift_tol;
      bool keep_net = !spot && valid, to_lbm = false;
      if (spot) {
        // the network's window error stands for the windows up to the next check
        const double e = sums[2 * T + 2 * a] / std::max(sums[2 * T + 2 * a + 1], 1e-300);
        R->trace[(size_t)i * maxJ + j] = flags[a] ? HUGE_VAL : e;
        const int ahead = anchor ? std::min(C - 1, J[i] - j - 1) : std::min(C, J[i] - j);
        est[i] += (std::isfinite(e) && !flags[a]) ? e * ahead : HUGE_VAL;
        checks[i] += 1;
        const bool over = !(est[i] <= R->cfg.l1_tol);
        if (anchor) {
          to_lbm = true;  // the LBM's window is kept
          if (over) fail_step[i] = (j + 1) * jump;
        } else {
          keep_net = valid && !over;
        }
      }
      if (keep_net) {
        windows[i] += 1;
        from_next.push_back(i);
      } else if (to_lbm) {
        from_lbm.push_back(i);
      } else if (anchor) {
        fail_step[i] = j * jump;  // the pre-window state stays
      } else {
        fail_step[i] = 0;  // the LBM runs the tube from its initial state
        from_init.push_back(i);
      }
    }
    // the window's start becomes the next window's previous state
    std::vector<int> kept(from_next);
    kept.insert(kept.end(), from_lbm.begin(), from_lbm.end());
    rpk_status st2 = copy_blocks(R, state, R->prev, kept, R->lists);
    if (st2 == RPK_OK) st2 = copy_blocks(R, R->next, state, from_next, R->lists);
    if (st2 == RPK_OK) st2 = copy_blocks(R, R->lbm, state, from_lbm, R->lists + T);
    if (st2 == RPK_OK) st2 = copy_blocks(R, R->init, state, from_init, R->lists);
    if (st2 != RPK_OK) return st2;
    for (int i : kept) has_prev[i] = 1;
  }
  // the LBM finishes every tube: fallback tubes from their last accepted state,
  // the others for their remainder steps
  bool any = false;
  std::vector<int> rest;
  for (int i = 0; i < T; ++i) {
    steps[i] = fail_step[i] >= 0 ? R->tubes[i].nsteps - fail_step[i] : R->tubes[i].nsteps - J[i] * jump;
    if (steps[i] > 0) {
      any = true;
      rest.push_back(i);
    }
  }
  if (any) {
    cudaEventRecord(R->ev[0], R->stream);
    rpk_status st = lbm_run(R, state, steps);
    if (st != RPK_OK) return st;
    cudaEventRecord(R->ev[1], R->stream);
    t_fb += elapsed(R);
    st = copy_blocks(R, R->lbm, state, rest, R->lists);
    if (st != RPK_OK) return st;
  }
  // a tube whose final moments are invalid is run again by the LBM from its
  // initial state
  std::vector<int> rerun(T, 0), again;
  {
    std::vector<rpk_sur_seq> hs(T);
    for (int i = 0; i < T; ++i) hs[i] = make_seq(R, i, 0);
    RPK_CUDA(cudaMemcpyAsync(R->seqs, hs.data(), sizeof(rpk_sur_seq) * T, cudaMemcpyHostToDevice, R->stream));
    k_valid<<<T, 256, 0, R->stream>>>(state, R->seqs, R->flags);
    RPK_CUDA(cudaGetLastError());
    RPK_CUDA(cudaMemcpyAsync(flags.data(), R->flags, sizeof(int) * T, cudaMemcpyDeviceToHost, R->stream));
    RPK_CUDA(cudaStreamSynchronize(R->stream));
    for (int i = 0; i < T; ++i)
      if (flags[i]) {
        rerun[i] = 1;
        again.push_back(i);
      }
  }
  double t_rerun = 0.0;
  if (!again.empty()) {
    std::vector<int> full(T, 0);
    for (int i : again) full[i] = R->tubes[i].nsteps;
    cudaEventRecord(R->ev[0], R->stream);
    rpk_status st = lbm_run(R, R->init, full);
    if (st != RPK_OK) return st;
    cudaEventRecord(R->ev[1], R->stream);
    t_rerun = elapsed(R);
    st = copy_blocks(R, R->lbm, state, again, R->lists);
    if (st != RPK_OK) return st;
  }
  RPK_CUDA(cudaStreamSynchronize(R->stream));
  if (stats)
    for (int i = 0; i < T; ++i) {
      stats[5 * i] = rerun[i] ? 0 : fail_step[i];
      stats[5 * i + 1] = windows[i];
      stats[5 * i + 2] = checks[i];
      stats[5 * i + 3] = rerun[i] ? R->tubes[i].nsteps : steps[i];
      stats[5 * i + 4] = rerun[i];
    }
  if (est_out)
    for (int i = 0; i < T; ++i) est_out[i] = est[i];
  if (ms) {
    ms[0] = t_net;
    ms[1] = t_spot;
    ms[2] = t_fb;
    ms[3] = t_rerun;
  }
  return RPK_OK;
}

rpk_status rpk_rollout_errors(const rpk_rollout* R, double* out, int* windows) {
  if (!R || !windows) return rpk::fail(RPK_ERR_ARG, "NULL argument");
  *windows = R->trace_windows;
  if (out && !R->trace.empty()) std::memcpy(out, R->trace.data(), sizeof(double) * R->trace.size());
  return RPK_OK;
}

}  // extern "C"
