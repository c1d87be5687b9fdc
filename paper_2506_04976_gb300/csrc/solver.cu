// Preconditioned proximal stochastic gradient solver (eq. 6) with the SGD, SAGA
// (eq. 7) and SVRG (eq. 9, Algorithm 1) estimators, the stepsize rules of Sec. 2.2 /
// Table 1 and the diagonal preconditioners of Sec. 2.3, driven epoch by epoch; each
// epoch is captured into a CUDA graph (one per epoch kind) and replayed after an
// in-place parameter update.
//
// Every subset function shares the same prior term (beta/n) S (eq. 5), so the prior
// part of the SAGA/SVRG estimator telescopes exactly:
//   n((beta/n) grad S(x) - (beta/n) grad S(xhat)) + beta grad S(xhat) = beta grad S(x).
// The gradient tables therefore hold data-term gradients only and the prior gradient
// is evaluated once per iteration at the current iterate.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pet_internal.cuh"
#include "pet_plan.h"

using namespace petgb;

namespace {

struct SolverState {  // device-resident scalars
  double tau_bb;
  int have_bb;
  int have_snapshot;
  double dots[2];     // p'q, q'q of the last refresh
};

struct UpdArgs {
  float *x;
  const float *D;
  float *g;          // subset data gradient (zeroed after use)
  const float *gS;   // beta grad S(x)
  float *table;      // [n][N] data gradients (SAGA/SVRG)
  float *G;          // sum of table
  size_t N;
  int n, subset;
  long long k;
  int rule;
  float tau0, eta;
  SolverState *st;
  double *tau_log;   // indexed by k (may be NULL)
};

__device__ __forceinline__ float step_of(const UpdArgs &a) {
  double tau;
  const double k = (double)a.k;
  switch (a.rule) {
    case PET_STEP_CONST: tau = a.tau0; break;
    case PET_STEP_VANISH: tau = a.tau0 / (1.0 + a.eta * k / a.n); break;
    case PET_STEP_ALG1:
      tau = a.k < 10 ? 3.0 : a.k < 100 ? 2.0 : a.k < 200 ? 1.5 : a.k < 300 ? 1.0 : 0.5;
      break;
    case PET_STEP_BB: tau = a.st->have_bb ? a.st->tau_bb : a.tau0; break;
    default: {
      const double bb = a.st->have_bb ? a.st->tau_bb : a.tau0;
      const double cap = a.k < 10 ? 3.0 : (a.k < 2LL * a.n ? 2.2 : 1.0);
      tau = bb < cap ? bb : cap;
    }
  }
  return (float)tau;
}

// ALGO: 0 SGD, 1 SAGA, 2 SVRG inner, 3 SVRG refresh (direction = full gradient).
template <int ALGO>
__global__ void k_update(UpdArgs a) {
  const float tau = step_of(a);
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.tau_log) a.tau_log[a.k] = tau;
  const float nf = (float)a.n;
  float *Ti = a.table ? a.table + (size_t)a.subset * a.N : nullptr;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < a.N; i += (size_t)gridDim.x * blockDim.x) {
    float dir;
    if (ALGO == 0) {
      dir = fmaf(nf, a.g[i], a.gS[i]);
      a.g[i] = 0.f;
    } else if (ALGO == 1) {
      const float gi = a.g[i], ti = Ti[i], Gi = a.G[i];
      dir = fmaf(nf, gi - ti, Gi) + a.gS[i];
      a.G[i] = Gi + (gi - ti);
      Ti[i] = gi;
      a.g[i] = 0.f;
    } else if (ALGO == 2) {
      dir = fmaf(nf, a.g[i] - Ti[i], a.G[i]) + a.gS[i];
      a.g[i] = 0.f;
    } else {
      dir = a.G[i] + a.gS[i];
    }
    const float xn = fmaf(-tau * a.D[i], dir, a.x[i]);
    a.x[i] = xn > 0.f ? xn : 0.f;
  }
}

// G = sum_s table[s]
__global__ void k_sum_table(const float *__restrict__ table, float *__restrict__ G, int n, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int t = 0; t < n; ++t) s += table[(size_t)t * N + i];
    G[i] = s;
  }
}

__device__ __forceinline__ double warp_block_sum(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// BB ingredients at an SVRG refresh, FP64: p = x - xhat_old, q = (G + gS) - Gfull_old;
// partial sums of p'q and q'q per block; then the snapshot buffers take the new values.
__global__ void k_bb_dots(const float *__restrict__ x, float *__restrict__ xhat_old,
                          const float *__restrict__ G, const float *__restrict__ gS,
                          float *__restrict__ Gfull_old, size_t N, double *part) {
  double pq = 0.0, qq = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const float gf = G[i] + gS[i];
    const double p = (double)x[i] - (double)xhat_old[i];
    const double q = (double)gf - (double)Gfull_old[i];
    pq += p * q;
    qq += q * q;
    xhat_old[i] = x[i];
    Gfull_old[i] = gf;
  }
  const double a = warp_block_sum(pq);
  if (threadIdx.x == 0) part[2 * blockIdx.x] = a;
  const double b = warp_block_sum(qq);
  if (threadIdx.x == 0) part[2 * blockIdx.x + 1] = b;
}

__global__ void k_bb_final(const double *part, int nb, SolverState *st) {
  if (threadIdx.x != 0) return;
  double pq = 0.0, qq = 0.0;
  for (int b = 0; b < nb; ++b) { pq += part[2 * b]; qq += part[2 * b + 1]; }
  st->dots[0] = pq;
  st->dots[1] = qq;
  if (st->have_snapshot && qq > 0.0) {
    st->tau_bb = pq / qq;
    st->have_bb = 1;
  }
  st->have_snapshot = 1;
}

unsigned grid_elems(size_t N) { return (unsigned)std::min<size_t>((size_t)152 * 8, (N + 255) / 256); }

uint64_t splitmix64(uint64_t &s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

}  // namespace

struct pet_solver {
  pet_plan *plan = nullptr;
  pet_solver_opts o;
  std::vector<long long> pc;
  std::vector<int> order;
  uint64_t rng = 0;
  std::vector<int> perm;
  long long k = 0;
  int n = 1;
  size_t N = 0;
  float *x = nullptr, *D = nullptr, *g = nullptr, *gS = nullptr, *H = nullptr;
  float *table = nullptr, *G = nullptr, *xhat_old = nullptr, *Gfull_old = nullptr;
  double *part = nullptr;
  int npart = 0;
  SolverState *st = nullptr;
  double *tau_log = nullptr;
  long long tau_cap = 0;
  bool initialised = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // [0] plain epoch, [1] epoch starting with a refresh
};

static pet_status grow_tau_log(pet_solver *s, long long need) {
  if (need <= s->tau_cap) return PET_OK;
  long long cap = std::max(need, 2 * s->tau_cap + 1024);
  double *nl = nullptr;
  if (cudaMalloc(&nl, cap * sizeof(double)) != cudaSuccess) return PET_ERR_NOMEM;
  cudaMemset(nl, 0, cap * sizeof(double));
  if (s->tau_log) {
    cudaMemcpy(nl, s->tau_log, s->tau_cap * sizeof(double), cudaMemcpyDeviceToDevice);
    cudaFree(s->tau_log);
  }
  s->tau_log = nl;
  s->tau_cap = cap;
  for (auto &e : s->exec)
    if (e) { cudaGraphExecDestroy(e); e = nullptr; }
  return PET_OK;
}

static void solver_free(pet_solver *s) {
  if (!s) return;
  for (auto &e : s->exec)
    if (e) cudaGraphExecDestroy(e);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  cudaFree(s->x); cudaFree(s->D); cudaFree(s->g); cudaFree(s->gS); cudaFree(s->H);
  cudaFree(s->table); cudaFree(s->G); cudaFree(s->xhat_old); cudaFree(s->Gfull_old);
  cudaFree(s->part); cudaFree(s->st); cudaFree(s->tau_log);
  delete s;
}

extern "C" pet_status pet_solver_create(pet_plan *plan, const pet_solver_opts *opts, pet_solver **out) {
  if (!plan || !opts || !out) return PET_ERR_ARG;
  *out = nullptr;
  if (!plan->has_data) return PET_ERR_STATE;
  const pet_solver_opts &o = *opts;
  if (o.algo < 0 || o.algo > 2 || o.step_rule < 0 || o.step_rule > 4 || o.precond_kind < 0 ||
      o.precond_kind > 1 || (o.algo == PET_SVRG && o.omega < 1) || (o.n_pc > 0 && !o.pc_iters) ||
      (o.norder > 0 && !o.order))
    return PET_ERR_ARG;
  pet_solver *s = new pet_solver();
  s->plan = plan;
  s->o = o;
  s->pc.assign(o.pc_iters, o.pc_iters + std::max(0, o.n_pc));
  if (o.norder > 0) s->order.assign(o.order, o.order + o.norder);
  for (int v : s->order)
    if (v < 0 || v >= plan->g.nsubsets) { delete s; return PET_ERR_ARG; }
  s->o.pc_iters = nullptr;
  s->o.order = nullptr;
  s->n = plan->g.nsubsets;
  s->N = plan->N;
  s->rng = o.seed;
  const size_t N = s->N;
  s->npart = 2 * (int)grid_elems(N);
  bool ok = cudaMalloc(&s->x, N * 4) == cudaSuccess && cudaMalloc(&s->D, N * 4) == cudaSuccess &&
            cudaMalloc(&s->g, N * 4) == cudaSuccess && cudaMalloc(&s->gS, N * 4) == cudaSuccess &&
            cudaMalloc(&s->H, N * 4) == cudaSuccess &&
            cudaMalloc(&s->part, s->npart * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->st, sizeof(SolverState)) == cudaSuccess;
  if (ok && o.algo != PET_SGD)
    ok = cudaMalloc(&s->table, N * 4 * (size_t)s->n) == cudaSuccess && cudaMalloc(&s->G, N * 4) == cudaSuccess;
  if (ok && o.algo == PET_SVRG)
    ok = cudaMalloc(&s->xhat_old, N * 4) == cudaSuccess && cudaMalloc(&s->Gfull_old, N * 4) == cudaSuccess;
  if (!ok) { solver_free(s); return PET_ERR_NOMEM; }
  if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    solver_free(s);
    return PET_ERR_CUDA;
  }
  *out = s;
  return PET_OK;
}

extern "C" void pet_solver_destroy(pet_solver *s) { solver_free(s); }

extern "C" const float *pet_solver_image(const pet_solver *s) { return s ? s->x : nullptr; }
extern "C" long long pet_solver_iteration(const pet_solver *s) { return s ? s->k : -1; }

extern "C" pet_status pet_solver_set_image(pet_solver *s, const float *x, void *stream) {
  if (!s || !x) return PET_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N = s->N;
  if (cudaMemcpyAsync(s->x, x, N * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(s->g, 0, N * 4, st) != cudaSuccess ||
      cudaMemsetAsync(s->D, 0, N * 4, st) != cudaSuccess ||
      cudaMemsetAsync(s->st, 0, sizeof(SolverState), st) != cudaSuccess ||
      cudaMemsetAsync(s->plan->d_gT, 0, N * 4, st) != cudaSuccess)
    return PET_ERR_CUDA;
  s->k = 0;
  s->rng = s->o.seed;
  s->initialised = false;
  return PET_OK;
}

extern "C" long long pet_solver_taus(const pet_solver *s, double *taus, long long cap) {
  if (!s || !taus) return 0;
  const long long n = std::min(cap, s->k);
  if (n > 0 && s->tau_log) cudaMemcpy(taus, s->tau_log, n * sizeof(double), cudaMemcpyDeviceToHost);
  return n;
}

// Subset of iteration k: explicit order or one splitmix64 Fisher-Yates permutation per epoch.
static int subset_of(pet_solver *s, long long k) {
  if (!s->order.empty()) return k < (long long)s->order.size() ? s->order[k] : -1;
  const int n = s->n;
  if (k % n == 0 || s->perm.empty()) {
    s->perm.resize(n);
    for (int i = 0; i < n; ++i) s->perm[i] = i;
    for (int i = n - 1; i >= 1; --i) {
      const int j = (int)(splitmix64(s->rng) % (uint64_t)(i + 1));
      std::swap(s->perm[i], s->perm[j]);
    }
  }
  return s->perm[k % n];
}

#define SCK(call)                                 \
  do {                                            \
    if ((call) != cudaSuccess) return PET_ERR_CUDA; \
  } while (0)

// Data gradient of subset `sub` at x into `dst` (zeroed by the caller unless deterministic).
static pet_status data_grad(pet_solver *s, int sub, float *dst, cudaStream_t st) {
  pet_plan *p = s->plan;
  if (s->o.deterministic) {
    pet_status e = pet_objective_grad(p, sub, s->x, dst, nullptr, nullptr, PET_GRAD_DETERMINISTIC, st);
    return e;
  }
  SCK(launch_grad(p->dp, sub, nullptr, s->x, p->d_xT, dst, p->d_gT, nullptr, MODE_GRAD, nullptr, st));
  SCK(launch_transpose(p->d_gT, dst, p->g.nx, p->g.ny, p->g.nz, 1, 2, st));  // add and clear
  return PET_OK;
}

static RdpArgs prior_args(const pet_solver *s, float scale) {
  pet_rdp_params rp;
  rp.nx = s->plan->g.nx; rp.ny = s->plan->g.ny; rp.nz = s->plan->g.nz;
  rp.dx = s->plan->g.dx; rp.dy = s->plan->g.dy; rp.dz = s->plan->g.dz;
  rp.gamma = s->o.gamma; rp.eps = s->o.eps; rp.scale = scale; rp.kappa = s->o.kappa;
  return make_rdp_args(rp);
}

static pet_status precond_update(pet_solver *s, cudaStream_t st) {
  pet_plan *p = s->plan;
  const bool harmonic = s->o.precond_kind == 1;
  if (harmonic) SCK(launch_rdp(prior_args(s, s->o.beta), s->x, nullptr, s->H, nullptr, 0, nullptr, st));
  SCK(launch_max(s->x, s->N, p->d_fpart, p->d_fscalar, st));
  SCK(launch_precond(s->x, p->d_sens, harmonic ? s->H : nullptr, (float)s->o.alpha, p->d_fscalar,
                     (float)s->o.delta_rel, s->D, s->N, st));
  return PET_OK;
}

static UpdArgs upd_args(pet_solver *s, int sub, long long k) {
  UpdArgs a;
  a.x = s->x; a.D = s->D; a.g = s->g; a.gS = s->gS; a.table = s->table; a.G = s->G;
  a.N = s->N; a.n = s->n; a.subset = sub < 0 ? 0 : sub; a.k = k;
  a.rule = s->o.step_rule; a.tau0 = (float)s->o.tau0; a.eta = (float)s->o.eta;
  a.st = s->st; a.tau_log = s->tau_log;
  return a;
}

// SAGA table initialisation: all entries at the start image (no step).
static pet_status saga_init(pet_solver *s, cudaStream_t st) {
  pet_plan *p = s->plan;
  SCK(to_frames(p, s->x, st));
  for (int t = 0; t < s->n; ++t) {
    float *Tt = s->table + (size_t)t * s->N;
    SCK(cudaMemsetAsync(Tt, 0, s->N * 4, st));
    pet_status e = data_grad(s, t, Tt, st);
    if (e != PET_OK) return e;
  }
  k_sum_table<<<grid_elems(s->N), 256, 0, st>>>(s->table, s->G, s->n, s->N);
  SCK(cudaGetLastError());
  return PET_OK;
}

// One iteration k of eq. 6 (Algorithm 1 for SVRG), enqueued on st.
static pet_status iterate(pet_solver *s, long long k, int sub, cudaStream_t st) {
  pet_plan *p = s->plan;
  for (long long c : s->pc)
    if (c == k) {
      pet_status e = precond_update(s, st);
      if (e != PET_OK) return e;
    }
  const unsigned ge = grid_elems(s->N);
  const bool refresh = s->o.algo == PET_SVRG && k % ((long long)s->o.omega * s->n) == 0;
  SCK(to_frames(p, s->x, st));
  if (refresh) {
    for (int t = 0; t < s->n; ++t) {
      float *Tt = s->table + (size_t)t * s->N;
      if (!s->o.deterministic) SCK(cudaMemsetAsync(Tt, 0, s->N * 4, st));
      pet_status e = data_grad(s, t, Tt, st);
      if (e != PET_OK) return e;
    }
    k_sum_table<<<ge, 256, 0, st>>>(s->table, s->G, s->n, s->N);
    SCK(launch_rdp(prior_args(s, s->o.beta), s->x, s->gS, nullptr, nullptr, 0, nullptr, st));
    k_bb_dots<<<ge, 256, 0, st>>>(s->x, s->xhat_old, s->G, s->gS, s->Gfull_old, s->N, s->part);
    k_bb_final<<<1, 32, 0, st>>>(s->part, (int)ge, s->st);
    k_update<3><<<ge, 256, 0, st>>>(upd_args(s, -1, k));
  } else {
    if (sub < 0) return PET_ERR_ARG;
    pet_status e = data_grad(s, sub, s->g, st);
    if (e != PET_OK) return e;
    SCK(launch_rdp(prior_args(s, s->o.beta), s->x, s->gS, nullptr, nullptr, 0, nullptr, st));
    const UpdArgs a = upd_args(s, sub, k);
    if (s->o.algo == PET_SGD) k_update<0><<<ge, 256, 0, st>>>(a);
    else if (s->o.algo == PET_SAGA) k_update<1><<<ge, 256, 0, st>>>(a);
    else k_update<2><<<ge, 256, 0, st>>>(a);
  }
  SCK(cudaGetLastError());
  return PET_OK;
}

static bool epoch_has_pc(const pet_solver *s, long long k0, long long len) {
  for (long long c : s->pc)
    if (c >= k0 && c < k0 + len) return true;
  return false;
}

extern "C" pet_status pet_solver_run(pet_solver *s, long long niter, void *stream) {
  if (!s || niter < 0) return PET_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!s->order.empty() && s->k + niter > (long long)s->order.size()) return PET_ERR_ARG;
  pet_status e = grow_tau_log(s, s->k + niter);
  if (e != PET_OK) return e;
  if (!s->initialised) {
    if (s->o.algo == PET_SAGA) {
      e = saga_init(s, st);
      if (e != PET_OK) return e;
    }
    s->initialised = true;
  }
  const long long end = s->k + niter;
  const int n = s->n;
  while (s->k < end) {
    const long long k0 = s->k;
    const bool whole_epoch = k0 % n == 0 && k0 + n <= end;
    if (s->o.use_graph && whole_epoch && !epoch_has_pc(s, k0, n) && !s->o.deterministic) {
      const int kind = (s->o.algo == PET_SVRG && k0 % ((long long)s->o.omega * n) == 0) ? 1 : 0;
      std::vector<int> subs(n);
      for (int j = 0; j < n; ++j) subs[j] = subset_of(s, k0 + j);
      cudaGraph_t graph = nullptr;
      SCK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
      pet_status ie = PET_OK;
      for (int j = 0; j < n && ie == PET_OK; ++j) ie = iterate(s, k0 + j, subs[j], s->cap_stream);
      cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &graph);
      if (ie != PET_OK) { if (graph) cudaGraphDestroy(graph); return ie; }
      if (ce != cudaSuccess) return PET_ERR_CUDA;
      bool updated = false;
      if (s->exec[kind]) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(s->exec[kind], graph, &info) == cudaSuccess;
        if (!updated) { cudaGetLastError(); cudaGraphExecDestroy(s->exec[kind]); s->exec[kind] = nullptr; }
      }
      if (!updated) {
        if (cudaGraphInstantiate(&s->exec[kind], graph, 0) != cudaSuccess) {
          cudaGraphDestroy(graph);
          return PET_ERR_CUDA;
        }
      }
      cudaGraphDestroy(graph);
      SCK(cudaGraphLaunch(s->exec[kind], st));
      s->k = k0 + n;
    } else {
      const int sub = subset_of(s, k0);
      e = iterate(s, k0, sub, st);
      if (e != PET_OK) return e;
      s->k = k0 + 1;
    }
  }
  return PET_OK;
}
