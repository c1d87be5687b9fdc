// Preconditioned proximal stochastic gradient solver (eq. 6) with the SGD, SAGA
// (eq. 7) and SVRG (eq. 9, Algorithm 1) estimators, the stepsize rules of Sec. 2.2 /
// Table 1 and the diagonal preconditioners of Sec. 2.3, driven epoch by epoch; each
// epoch is captured into a CUDA graph (one per epoch kind) and replayed after an
// in-place parameter update.
//
// Every subset function shares the same prior term (beta/n) S (eq. 5).  In SVRG all
// table entries belong to one snapshot xhat, so the prior part of eq. 9 telescopes
// exactly:  n((beta/n) grad S(x) - (beta/n) grad S(xhat)) + beta grad S(xhat) = beta grad S(x);
// the SVRG table therefore holds data-term gradients only.  SAGA's entries come from
// different iterates and do not telescope, so its table holds full subset gradients
// grad f_i = grad D_i + (beta/n) grad S, exactly as eq. 7 states.  The prior gradient
// beta grad S(x) is evaluated once per iteration at the current iterate.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdlib>
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
  float *x, *xT;     // iterate, canonical [z][y][x] and transposed [z][x][y]
  const float *D;
  const float *g, *gT;  // subset data gradient: canonical part and transposed part
                        // (x-driven views)
  const float *gS;   // beta grad S(x)
  float *table;      // [n][N] data gradients (SAGA/SVRG)
  float *G;          // sum of table
  int nx, ny, nz;
  size_t N;
  int n, subset;
  long long k;
  int rule;
  float tau0, eta;
  SolverState *st;
  double *tau_log;   // indexed by k (may be NULL)
  const int *subset_dev;     // if set, the subset is read from device memory (batches)
  const long long *k_dev;    // if set, the iteration index is read from device memory
  const float *w_dev;        // SVRG: weight 1/p_i of the sampled subset (NULL: n)
  const float *gSh;          // SVRG with non-uniform weights: beta grad S(xhat) (else NULL)
  int *sub_log;              // indexed by k: subset used, -1 at SVRG refreshes (may be NULL)
};

__device__ __forceinline__ float step_of(const UpdArgs &a, long long ki) {
  double tau;
  const double k = (double)ki;
  switch (a.rule) {
    case PET_STEP_CONST: tau = a.tau0; break;
    case PET_STEP_VANISH: tau = a.tau0 / (1.0 + a.eta * k / a.n); break;
    case PET_STEP_ALG1:
      tau = ki < 10 ? 3.0 : ki < 100 ? 2.0 : ki < 200 ? 1.5 : ki < 300 ? 1.0 : 0.5;
      break;
    case PET_STEP_BB: tau = a.st->have_bb ? a.st->tau_bb : a.tau0; break;
    default: {
      const double bb = a.st->have_bb ? a.st->tau_bb : a.tau0;
      const double cap = ki < 10 ? 3.0 : (ki < 2LL * a.n ? 2.2 : 1.0);
      tau = bb < cap ? bb : cap;
    }
  }
  return (float)tau;
}

// Fused estimator + preconditioned step + prox (eq. 6 with eq. 7 / eq. 9) on a 32x32
// tile of one slice.  The transposed gradient part is read through shared memory; the
// new iterate is written in both layouts.  The gradient accumulators are cleared
// afterwards by k_clear2 (clearing them here, with scalar stores into lines that the
// projector's atomics just updated, measured about three times slower).  The stepsize is evaluated once
// per block.  ALGO: 0 SGD, 1 SAGA, 2 SVRG inner, 3 SVRG refresh (direction = full
// gradient at the snapshot).
template <int ALGO>
__device__ __forceinline__ void upd_body(const UpdArgs &a, int bx, int by, int z) {
  __shared__ float tin[32][33];
  __shared__ float tout[32][33];
  __shared__ float s_tau, s_w;
  __shared__ int s_sub;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = bx * 32, y0 = by * 32;
  const size_t sl = (size_t)z * a.nx * a.ny;
  if (tx == 0 && ty == 0) {
    const long long k = a.k_dev ? *a.k_dev : a.k;
    s_tau = step_of(a, k);
    s_sub = a.subset_dev ? *a.subset_dev : a.subset;
    s_w = a.w_dev ? *a.w_dev : (float)a.n;
    if (bx == 0 && by == 0 && z == 0) {
      if (a.tau_log) a.tau_log[k] = s_tau;
      if (a.sub_log) a.sub_log[k] = ALGO == 3 ? -1 : s_sub;
    }
  }
  if (ALGO != 3) {
    for (int j = ty; j < 32; j += 8) {
      const int xx = x0 + j, yy = y0 + tx;
      float v = 0.f;
      if (xx < a.nx && yy < a.ny) v = a.gT[sl + (size_t)xx * a.ny + yy];
      tin[j][tx] = v;
    }
  }
  __syncthreads();
  const float tau = s_tau;
  const float nf = (float)a.n;
  float *Ti = a.table ? a.table + (size_t)s_sub * a.N : nullptr;
  for (int j = ty; j < 32; j += 8) {
    const int xx = x0 + tx, yy = y0 + j;
    float xn = 0.f;
    if (xx < a.nx && yy < a.ny) {
      const size_t i = sl + (size_t)yy * a.nx + xx;
      float dir;
      if (ALGO == 3) {
        dir = a.G[i] + a.gS[i];
      } else {
        const float gi = a.g[i] + tin[tx][j];
        if (ALGO == 0) {
          dir = fmaf(nf, gi, a.gS[i]);
        } else if (ALGO == 1) {
          const float gf = fmaf(a.gS[i], 1.f / nf, gi);  // grad f_i = grad D_i + (beta/n) grad S
          const float ti = Ti[i], Gi = a.G[i];
          dir = fmaf(nf, gf - ti, Gi);
          a.G[i] = Gi + (gf - ti);
          Ti[i] = gf;
        } else {
          // SVRG, eq. 9: w (grad D_i(x) - grad D_i(xhat)) + grad D(xhat) + beta grad S(x), the
          // prior part telescoped for w = n; a table-free solver's g already holds the
          // difference.  For w != n the prior part is (w/n)(gS - gSh) + gSh exactly.
          const float w = s_w;
          dir = fmaf(w, Ti ? gi - Ti[i] : gi, a.G[i]) + a.gS[i];
          if (a.gSh) dir = fmaf(w / nf - 1.f, a.gS[i] - a.gSh[i], dir);
        }
      }
      xn = fmaf(-tau * a.D[i], dir, a.x[i]);
      xn = xn > 0.f ? xn : 0.f;
      a.x[i] = xn;
    }
    tout[tx][j] = xn;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int xx = x0 + j, yy = y0 + tx;
    if (xx < a.nx && yy < a.ny) a.xT[sl + (size_t)xx * a.ny + yy] = tout[j][tx];
  }
}

// The same update for images larger than the L2 share of the step (every operand comes
// from HBM): a thread first issues the loads of all four of its rows (and of the
// transposed gradient part), then computes and stores, so that more bytes are in flight
// per thread.  Results are identical to upd_body.
template <int ALGO>
__device__ __forceinline__ void upd_body_ilp(const UpdArgs &a, int bx, int by, int z) {
  __shared__ float tin[32][33];
  __shared__ float tout[32][33];
  __shared__ float s_tau, s_w;
  __shared__ int s_sub;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = bx * 32, y0 = by * 32;
  const size_t sl = (size_t)z * a.nx * a.ny;
  if (tx == 0 && ty == 0) {
    const long long k = a.k_dev ? *a.k_dev : a.k;
    s_tau = step_of(a, k);
    s_sub = a.subset_dev ? *a.subset_dev : a.subset;
    s_w = a.w_dev ? *a.w_dev : (float)a.n;
    if (bx == 0 && by == 0 && z == 0) {
      if (a.tau_log) a.tau_log[k] = s_tau;
      if (a.sub_log) a.sub_log[k] = ALGO == 3 ? -1 : s_sub;
    }
  }
  // the subset (table entry) is known to thread 0 only before the barrier; every other
  // operand is loaded now
  constexpr int R = 4;  // rows per thread
  bool in[R];
  size_t idx[R];
  float gv[R], sv[R], Dv[R], xv[R], Gv[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int xx = x0 + tx, yy = y0 + ty + 8 * q;
    in[q] = xx < a.nx && yy < a.ny;
    idx[q] = in[q] ? sl + (size_t)yy * a.nx + xx : 0;
    gv[q] = (ALGO != 3 && in[q]) ? a.g[idx[q]] : 0.f;
    sv[q] = in[q] ? a.gS[idx[q]] : 0.f;
    Dv[q] = in[q] ? a.D[idx[q]] : 0.f;
    xv[q] = in[q] ? a.x[idx[q]] : 0.f;
    Gv[q] = (ALGO != 0 && in[q]) ? a.G[idx[q]] : 0.f;
  }
  if (ALGO != 3) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int j = ty + 8 * q;
      const int xx = x0 + j, yy = y0 + tx;
      float v = 0.f;
      if (xx < a.nx && yy < a.ny) v = a.gT[sl + (size_t)xx * a.ny + yy];
      tin[j][tx] = v;
    }
  }
  __syncthreads();
  const float tau = s_tau;
  const float nf = (float)a.n;
  float *Ti = a.table ? a.table + (size_t)s_sub * a.N : nullptr;
  float tv[R], hv[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    tv[q] = ((ALGO == 1 || ALGO == 2) && Ti && in[q]) ? Ti[idx[q]] : 0.f;
    hv[q] = (ALGO == 2 && a.gSh && in[q]) ? a.gSh[idx[q]] : 0.f;
  }
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int j = ty + 8 * q;
    float xn = 0.f;
    if (in[q]) {
      float dir;
      if (ALGO == 3) {
        dir = Gv[q] + sv[q];
      } else {
        const float gi = gv[q] + tin[tx][j];
        if (ALGO == 0) {
          dir = fmaf(nf, gi, sv[q]);
        } else if (ALGO == 1) {
          const float gf = fmaf(sv[q], 1.f / nf, gi);
          dir = fmaf(nf, gf - tv[q], Gv[q]);
          a.G[idx[q]] = Gv[q] + (gf - tv[q]);
          Ti[idx[q]] = gf;
        } else {
          const float w = s_w;
          dir = fmaf(w, Ti ? gi - tv[q] : gi, Gv[q]) + sv[q];
          if (a.gSh) dir = fmaf(w / nf - 1.f, sv[q] - hv[q], dir);
        }
      }
      xn = fmaf(-tau * Dv[q], dir, xv[q]);
      xn = xn > 0.f ? xn : 0.f;
      a.x[idx[q]] = xn;
    }
    tout[tx][j] = xn;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int xx = x0 + j, yy = y0 + tx;
    if (xx < a.nx && yy < a.ny) a.xT[sl + (size_t)xx * a.ny + yy] = tout[j][tx];
  }
}

template <int ALGO>
__global__ void __launch_bounds__(256) k_update(UpdArgs a) {
  upd_body<ALGO>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int ALGO>
__global__ void __launch_bounds__(256) k_update_ilp(UpdArgs a) {
  upd_body_ilp<ALGO>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Images whose update operands (six or seven image-sized arrays) exceed about half of the
// L2 cache take the variant with all loads issued first.
constexpr size_t kUpdIlpVoxels = (size_t)2 << 20;

// Job of this block among consecutive block ranges [begin[j], begin[j+1]).
__device__ __forceinline__ int batch_job(const int *__restrict__ begin, int njobs) {
  __shared__ int s_job;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid < 32) {
    int job = 0;
    for (int base = 0; base < njobs; base += 32) {
      const int j = base + tid;
      const unsigned m = __ballot_sync(0xffffffffu, j < njobs && __ldg(&begin[j]) <= (int)blockIdx.x);
      job = base + __popc(m) - 1;
      if (m != 0xffffffffu) break;
    }
    if (tid == 0) s_job = job;
  }
  __syncthreads();
  return s_job;
}

// Batched update: each job's blocks tile its image (32x32 tiles per slice).
template <int ALGO>
__global__ void __launch_bounds__(256) k_update_batch(const UpdArgs *__restrict__ jobs, const int *__restrict__ begin,
                                                      int njobs) {
  __shared__ UpdArgs sa;
  const int j = batch_job(begin, njobs);
  if (threadIdx.x == 0 && threadIdx.y == 0) sa = jobs[j];
  __syncthreads();
  if (*sa.subset_dev == kBatchSkip) return;  // this instance runs the window alone (whole block)
  const int blk = (int)blockIdx.x - __ldg(&begin[j]);
  const int tx = (sa.nx + 31) / 32, ty = (sa.ny + 31) / 32;
  upd_body<ALGO>(sa, blk % tx, (blk / tx) % ty, blk / (tx * ty));
}

struct ClearJob {
  float *a, *b;
  size_t N;
};

__global__ void __launch_bounds__(256) k_clear_batch(const ClearJob *__restrict__ jobs, const int *__restrict__ begin,
                                                     int njobs, const int *__restrict__ sub) {
  const int j = batch_job(begin, njobs);
  if (sub && __ldg(&sub[j]) == kBatchSkip) return;  // whole block: one job
  const ClearJob c = jobs[j];
  const int b0 = __ldg(&begin[j]), nb = __ldg(&begin[j + 1]) - b0;
  const size_t n4 = c.N / 4;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (size_t i = (size_t)(blockIdx.x - b0) * blockDim.x + threadIdx.x; i < n4; i += (size_t)nb * blockDim.x) {
    reinterpret_cast<float4 *>(c.a)[i] = z;
    reinterpret_cast<float4 *>(c.b)[i] = z;
  }
  for (size_t i = 4 * n4 + (size_t)(blockIdx.x - b0) * blockDim.x + threadIdx.x; i < c.N; i += (size_t)nb * blockDim.x) {
    c.a[i] = 0.f;
    c.b[i] = 0.f;
  }
}

// Zeroes one or two (b != NULL) image-sized accumulators with 16-byte stores (N must be a multiple of 4
// for the vector part; the tail is cleared element-wise).
__global__ void k_clear2(float *__restrict__ a, float *__restrict__ b, size_t N) {
  const size_t n4 = N / 4;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    reinterpret_cast<float4 *>(a)[i] = z;
    if (b) reinterpret_cast<float4 *>(b)[i] = z;
  }
  for (size_t i = 4 * n4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    a[i] = 0.f;
    if (b) b[i] = 0.f;
  }
}

// G = sum_s table[s]; with gS != NULL every entry first receives the prior share
// gS/n (SAGA's full subset gradients).
__global__ void k_sum_table(float *__restrict__ table, float *__restrict__ G, const float *__restrict__ gS,
                            int n, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const float pr = gS ? gS[i] * (1.f / (float)n) : 0.f;
    float s = 0.f;
    for (int t = 0; t < n; ++t) {
      float v = table[(size_t)t * N + i];
      if (gS) {
        v += pr;
        table[(size_t)t * N + i] = v;
      }
      s += v;
    }
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
// partial sums of p'q and q'Dq per block (the short BB step in the metric of the
// preconditioner D, so that it is on the scale of the other step rules, which also
// multiply D grad); then the snapshot buffers take the new values.
__global__ void k_bb_dots(const float *__restrict__ x, float *__restrict__ xhat_old,
                          const float *__restrict__ G, const float *__restrict__ gS,
                          float *__restrict__ Gfull_old, const float *__restrict__ D, size_t N, double *part) {
  double pq = 0.0, qq = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const float gf = G[i] + gS[i];
    const double p = (double)x[i] - (double)xhat_old[i];
    const double q = (double)gf - (double)Gfull_old[i];
    pq += p * q;
    qq += q * (double)D[i] * q;
    xhat_old[i] = x[i];
    Gfull_old[i] = gf;
  }
  const double a = warp_block_sum(pq);
  if (threadIdx.x == 0) part[2 * blockIdx.x] = a;
  const double b = warp_block_sum(qq);
  if (threadIdx.x == 0) part[2 * blockIdx.x + 1] = b;
}

__global__ void k_bb_final(const double *part, int nb, SolverState *st, int update) {
  double pq = 0.0, qq = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) { pq += part[2 * b]; qq += part[2 * b + 1]; }
  pq = warp_block_sum(pq);
  qq = warp_block_sum(qq);
  if (threadIdx.x != 0) return;
  st->dots[0] = pq;
  st->dots[1] = qq;
  if (update && st->have_snapshot && qq > 0.0) {
    st->tau_bb = pq / qq;
    st->have_bb = 1;
  }
  st->have_snapshot = 1;
}

// Importance sampling at an SVRG refresh (Sec. 2.4): FP64 partial sums of
// ||g_t + gS/n||^2 for subset t = blockIdx.y, over a grid-stride share of the image.
// src is the table entry of t (table == true) or an image-sized accumulator holding
// grad D_t (table == false), which is then added into G and cleared.
__global__ void k_sub_norms(float *__restrict__ src, const float *__restrict__ gS, float *__restrict__ G,
                            int n, size_t N, int from_table, double *__restrict__ part) {
  const int t = blockIdx.y;
  float *g = from_table ? src + (size_t)t * N : src;
  double acc = 0.0;
  const float inv_n = 1.f / (float)n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const float v = g[i];
    const double f = (double)fmaf(gS[i], inv_n, v);
    acc += f * f;
    if (!from_table) {
      G[i] += v;
      g[i] = 0.f;
    }
  }
  const double b = warp_block_sum(acc);
  if (threadIdx.x == 0) part[(size_t)t * gridDim.x + blockIdx.x] = b;
}

// p_t = ||grad f_t|| / sum_j ||grad f_j|| from the partial sums (uniform if all vanish).
__global__ void k_probs(const double *__restrict__ part, int nb, int n, double *__restrict__ prob) {
  __shared__ double nrm[1024];
  for (int t = 0; t < n; ++t) {
    double sacc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) sacc += part[(size_t)t * nb + b];
    sacc = warp_block_sum(sacc);
    if (threadIdx.x == 0) nrm[t] = sqrt(sacc);
  }
  if (threadIdx.x != 0) return;
  double tot = 0.0;
  for (int t = 0; t < n; ++t) tot += nrm[t];
  for (int t = 0; t < n; ++t) prob[t] = tot > 0.0 ? nrm[t] / tot : 1.0 / n;
}

// Importance draw of iteration k: u = (z >> 11) 2^-53 with z the k-th output of the
// splitmix64 stream from `seed`; the subset is the smallest t with u below the FP64
// cumulative sum of p (the last t with p_t > 0 if rounding leaves u above the sum).
__global__ void k_draw(const double *__restrict__ prob, int n, unsigned long long seed, long long k,
                       int *__restrict__ sub, float *__restrict__ w) {
  if (threadIdx.x != 0) return;
  unsigned long long z = seed + (unsigned long long)(k + 1) * 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  z = z ^ (z >> 31);
  const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  double c = 0.0;
  int pick = -1, last = 0;
  for (int t = 0; t < n; ++t) {
    const double pt = prob[t];
    if (pt > 0.0) last = t;
    c += pt;
    if (pick < 0 && pt > 0.0 && u < c) pick = t;
  }
  if (pick < 0) pick = last;
  *sub = pick;
  *w = (float)(1.0 / prob[pick]);
}

unsigned grid_elems(size_t N) { return (unsigned)std::min<size_t>((size_t)152 * 8, (N + 255) / 256); }

uint64_t splitmix64(uint64_t &s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Herman-Meyer order (Sec. 2.4): with the prime factors p1 <= p2 <= ... of n, epoch
// position j, written in mixed radix with its lowest digit in base p1, visits the subset
// whose digits are weighted n/p1, n/(p1 p2), ... (bit reversal when n is a power of 2).
std::vector<int> herman_meyer(int n) {
  std::vector<int> f;
  int r = n;
  for (int q = 2; q <= r; ++q)
    while (r % q == 0) { f.push_back(q); r /= q; }
  std::vector<int> out(n);
  for (int j = 0; j < n; ++j) {
    int rest = j, w = n, idx = 0;
    for (int p : f) {
      w /= p;
      idx += (rest % p) * w;
      rest /= p;
    }
    out[j] = idx;
  }
  return out;
}

// Cofactor order (Sec. 2.4): generators g of Z_n (gcd(g, n) = 1), nearest to 0.3 n or
// 0.7 n first (distance compared as min(|10 g - 3 n|, |10 g - 7 n|), ties to the smaller g).
std::vector<int> cofactor_generators(int n) {
  std::vector<int> g;
  for (int c = 1; c < n; ++c) {
    int a = c, b = n;
    while (b) { const int t = a % b; a = b; b = t; }
    if (a == 1) g.push_back(c);
  }
  auto dist = [n](int c) { return std::min(std::abs(10 * c - 3 * n), std::abs(10 * c - 7 * n)); };
  std::stable_sort(g.begin(), g.end(), [&](int a, int b) { return dist(a) < dist(b); });
  return g;
}

constexpr int kNormBlocks = 64;

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
  int *sub_log = nullptr;   // subset of every iteration, -1 at SVRG refreshes
  long long tau_cap = 0;
  // sampling rules of Sec. 2.4
  std::vector<int> hm;      // Herman-Meyer order
  std::vector<int> gens;    // cofactor generators, ranked
  // importance sampling (SVRG): probabilities, their partial sums, the drawn subset and
  // its weight, and beta grad S at the snapshot
  double *prob = nullptr, *norm_part = nullptr;
  int *d_sub = nullptr;
  float *d_w = nullptr, *gSh = nullptr;
  // table-free SVRG: the snapshot in the transposed layout (xhat_old holds the canonical one)
  float *xhatT = nullptr;
  bool initialised = false;
  cudaStream_t cap_stream = nullptr;
  // The prior's gradient depends only on x, so each iteration computes it on a second
  // stream, forked after the previous update and joined before the next one; its blocks
  // fill the SMs that the subset-gradient launch leaves idle in its last wave.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // Inner-iteration gradient accumulators (canonical, transposed), alternating with the
  // iteration's parity: while iteration k accumulates into one pair, the side stream
  // clears the pair iteration k-1 used (gbuf[0] is g).
  float *gbuf[2] = {nullptr, nullptr}, *gTbuf[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // [0] plain epoch, [1] epoch starting with a refresh
  // optional event timing of the fused subset-gradient kernel: one (start, stop) pair per
  // launch slot of an SVRG outer loop (or of an epoch for SGD/SAGA)
  bool profile = false;
  std::vector<cudaEvent_t> ev0, ev1;
  std::vector<char> pending;
  std::vector<int> kind_slots[2];
  double prof_ms = 0.0;
  long long prof_n = 0;
  int capturing_kind = 0;
};

static pet_status grow_tau_log(pet_solver *s, long long need) {
  if (need <= s->tau_cap) return PET_OK;
  // Rare (capacity doubles): wait for every launch that may still write the old logs,
  // whatever stream the caller used, before copying them.
  if (cudaDeviceSynchronize() != cudaSuccess) return PET_ERR_CUDA;
  long long cap = std::max(need, 2 * s->tau_cap + 1024);
  double *nl = nullptr;
  int *ns = nullptr;
  if (cudaMalloc(&nl, cap * sizeof(double)) != cudaSuccess) return PET_ERR_NOMEM;
  if (cudaMalloc(&ns, cap * sizeof(int)) != cudaSuccess) { cudaFree(nl); return PET_ERR_NOMEM; }
  bool ok = cudaMemset(nl, 0, cap * sizeof(double)) == cudaSuccess &&
            cudaMemset(ns, 0xff, cap * sizeof(int)) == cudaSuccess;
  if (ok && s->tau_log)
    ok = cudaMemcpy(nl, s->tau_log, s->tau_cap * sizeof(double), cudaMemcpyDeviceToDevice) == cudaSuccess &&
         cudaMemcpy(ns, s->sub_log, s->tau_cap * sizeof(int), cudaMemcpyDeviceToDevice) == cudaSuccess;
  if (!ok) { cudaFree(nl); cudaFree(ns); return PET_ERR_CUDA; }
  if (s->tau_log) {
    cudaFree(s->tau_log);
    cudaFree(s->sub_log);
  }
  s->tau_log = nl;
  s->sub_log = ns;
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
  if (s->side) cudaStreamDestroy(s->side);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  for (auto e : s->ev0) cudaEventDestroy(e);
  for (auto e : s->ev1) cudaEventDestroy(e);
  cudaFree(s->x); cudaFree(s->D); cudaFree(s->g); cudaFree(s->gS); cudaFree(s->H);
  cudaFree(s->sub_log); cudaFree(s->prob); cudaFree(s->norm_part); cudaFree(s->d_sub); cudaFree(s->d_w);
  cudaFree(s->gSh); cudaFree(s->xhatT);
  cudaFree(s->gbuf[1]); cudaFree(s->gTbuf[0]); cudaFree(s->gTbuf[1]);
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
      (o.norder > 0 && !o.order) || o.sampling < PET_SAMPLE_PERM || o.sampling > PET_SAMPLE_IMPORTANCE ||
      ((o.sampling == PET_SAMPLE_IMPORTANCE || o.low_memory) && o.algo != PET_SVRG))
    return PET_ERR_ARG;
  if ((o.sampling == PET_SAMPLE_IMPORTANCE || o.low_memory) && o.deterministic) return PET_ERR_UNSUPPORTED;
  if (o.sampling == PET_SAMPLE_IMPORTANCE && plan->g.nsubsets > 1024) return PET_ERR_UNSUPPORTED;
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
    ok = (o.low_memory || cudaMalloc(&s->table, N * 4 * (size_t)s->n) == cudaSuccess) &&
         cudaMalloc(&s->G, N * 4) == cudaSuccess;
  if (ok && o.algo == PET_SVRG)
    ok = cudaMalloc(&s->xhat_old, N * 4) == cudaSuccess && cudaMalloc(&s->Gfull_old, N * 4) == cudaSuccess;
  if (ok) {
    s->gbuf[0] = s->g;
    ok = cudaMalloc(&s->gbuf[1], N * 4) == cudaSuccess && cudaMalloc(&s->gTbuf[0], N * 4) == cudaSuccess &&
         cudaMalloc(&s->gTbuf[1], N * 4) == cudaSuccess;
  }
  if (ok && o.low_memory) ok = cudaMalloc(&s->xhatT, N * 4) == cudaSuccess;
  if (ok && o.sampling == PET_SAMPLE_IMPORTANCE)
    ok = cudaMalloc(&s->prob, s->n * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&s->norm_part, (size_t)s->n * kNormBlocks * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&s->d_sub, sizeof(int)) == cudaSuccess && cudaMalloc(&s->d_w, sizeof(float)) == cudaSuccess &&
         cudaMalloc(&s->gSh, N * 4) == cudaSuccess;
  if (ok && o.sampling == PET_SAMPLE_HM) s->hm = herman_meyer(s->n);
  if (ok && o.sampling == PET_SAMPLE_COFACTOR) s->gens = cofactor_generators(s->n);
  if (!ok) { solver_free(s); return PET_ERR_NOMEM; }
  if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess) {
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
      cudaMemsetAsync(s->plan->d_gT, 0, N * 4, st) != cudaSuccess ||
      cudaMemsetAsync(s->gbuf[1], 0, N * 4, st) != cudaSuccess ||
      cudaMemsetAsync(s->gTbuf[0], 0, N * 4, st) != cudaSuccess ||
      cudaMemsetAsync(s->gTbuf[1], 0, N * 4, st) != cudaSuccess)
    return PET_ERR_CUDA;
  s->k = 0;
  s->rng = s->o.seed;
  s->initialised = false;
  return PET_OK;
}

extern "C" long long pet_solver_subsets(const pet_solver *s, int *subsets, long long cap) {
  if (!s || !subsets) return 0;
  const long long n = std::min(cap, s->k);
  if (n > 0 && s->sub_log && cudaMemcpy(subsets, s->sub_log, n * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return 0;
  return n;
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
  switch (s->o.sampling) {
    case PET_SAMPLE_REPLACE: {  // output k of the splitmix64 stream from the seed
      uint64_t st = s->o.seed + (uint64_t)k * 0x9e3779b97f4a7c15ULL;
      return (int)(((splitmix64(st) >> 32) * (uint64_t)n) >> 32);
    }
    case PET_SAMPLE_HM: return s->hm[k % n];
    case PET_SAMPLE_COFACTOR: {
      if (s->gens.empty()) return 0;
      const long long g = s->gens[(k / n) % (long long)s->gens.size()];
      return (int)(((k % n) * g) % n);
    }
    case PET_SAMPLE_IMPORTANCE: return 0;  // drawn on the device
    default: break;
  }
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

static int n_slots(const pet_solver *s) {
  return s->o.algo == PET_SVRG ? s->n + s->o.omega * s->n : s->n;
}

// Launch slot of the subset-gradient kernel: unique within one SVRG outer loop
// (refresh gradients 0..n-1, inner iterations after them) or one SGD/SAGA epoch.
static int slot_of(const pet_solver *s, long long k, int refresh_sub) {
  if (s->o.algo == PET_SVRG) {
    const long long kk = k % ((long long)s->o.omega * s->n);
    return refresh_sub >= 0 ? refresh_sub : (int)(s->n + kk - 1);
  }
  return (int)(k % s->n);
}

static cudaError_t record(pet_solver *s, cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  return cudaEventRecordWithFlags(ev, st, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                               : cudaEventRecordDefault);
}

// Data gradient of subset `sub` at x into `dst` (zeroed by the caller unless deterministic).
// sub_dev (may be NULL) supplies the subset from device memory; img/imgT (default: the
// iterate in both layouts) and mode (MODE_NGRAD subtracts) serve the table-free SVRG.
static pet_status data_grad(pet_solver *s, int sub, float *dst, cudaStream_t st, int slot = -1,
                            bool combine = true, const int *sub_dev = nullptr, const float *img = nullptr,
                            const float *imgT = nullptr, int mode = MODE_GRAD, float *dstT = nullptr) {
  pet_plan *p = s->plan;
  if (!dstT) dstT = p->d_gT;
  if (s->o.deterministic) {
    pet_status e = pet_objective_grad(p, sub, s->x, dst, nullptr, nullptr, PET_GRAD_DETERMINISTIC, st);
    return e;
  }
  const float *im = img ? img : s->x, *imT = imgT ? imgT : p->d_xT;
  if (p->res) {  // the projector reads G x (both layouts rebuilt from the canonical image)
    SCK(prepare_image(p, im, &im, st));
    imT = p->d_xT;
  }
  const bool prof = s->profile && slot >= 0 && slot < (int)s->ev0.size();
  if (prof) SCK(record(s, s->ev0[slot], st));
  SCK(launch_grad(p->dp, sub, sub_dev, im, imT, dst, dstT, nullptr, mode, nullptr, st));
  if (prof) {
    SCK(record(s, s->ev1[slot], st));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive) s->kind_slots[s->capturing_kind].push_back(slot);
    else s->pending[slot] = 1;
  }
  if (combine) {
    SCK(launch_transpose(dstT, dst, p->g.nx, p->g.ny, p->g.nz, 1, 1, st));  // add
    note_launch();
    k_clear2<<<grid_elems(s->N / 4), 256, 0, st>>>(dstT, nullptr, s->N);
    SCK(apply_res(p, dst, st));
  }
  return PET_OK;
}

static RdpArgs prior_args(const pet_solver *s, float scale) {
  pet_rdp_params rp;
  rp.nx = s->plan->g.nx; rp.ny = s->plan->g.ny; rp.nz = s->plan->g.nz;
  rp.dx = s->plan->g.dx; rp.dy = s->plan->g.dy; rp.dz = s->plan->g.dz;
  rp.gamma = s->o.gamma; rp.eps = s->o.eps; rp.scale = scale; rp.kappa = s->o.kappa;
  RdpArgs a = make_rdp_args(rp);
  a.zch = s->plan->rdp_zch;
  return a;
}

// grad S(x) into gS on the side stream, ordered after everything enqueued on st so far;
// join_prior makes st wait for it.  Under stream capture the two become graph branches.
static pet_status fork_prior(pet_solver *s, cudaStream_t st, int clear_buf) {
  SCK(cudaEventRecord(s->ev_fork, st));
  SCK(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
  SCK(launch_rdp(prior_args(s, s->o.beta), s->x, s->gS, nullptr, nullptr, 0, nullptr, s->side));
  note_launch();
  k_clear2<<<grid_elems(s->N / 4), 256, 0, s->side>>>(s->gbuf[clear_buf], s->gTbuf[clear_buf], s->N);
  SCK(cudaEventRecord(s->ev_join, s->side));
  return PET_OK;
}

static pet_status join_prior(pet_solver *s, cudaStream_t st) {
  SCK(cudaStreamWaitEvent(st, s->ev_join, 0));
  return PET_OK;
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
  pet_plan *p = s->plan;
  a.x = s->x; a.xT = p->d_xT; a.D = s->D; a.g = s->g; a.gT = p->d_gT; a.gS = s->gS;
  a.table = s->table; a.G = s->G;
  a.nx = p->g.nx; a.ny = p->g.ny; a.nz = p->g.nz;
  a.N = s->N; a.n = s->n; a.subset = sub < 0 ? 0 : sub; a.k = k;
  a.rule = s->o.step_rule; a.tau0 = (float)s->o.tau0; a.eta = (float)s->o.eta;
  a.st = s->st; a.tau_log = s->tau_log;
  a.subset_dev = s->d_sub;
  a.k_dev = nullptr;
  a.w_dev = s->d_w;
  a.gSh = s->gSh;
  a.sub_log = s->sub_log;
  return a;
}

static dim3 tile_grid(const pet_solver *s) {
  const pet_geometry &g = s->plan->g;
  return dim3((g.nx + 31) / 32, (g.ny + 31) / 32, g.nz);
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
  SCK(launch_rdp(prior_args(s, s->o.beta), s->x, s->gS, nullptr, nullptr, 0, nullptr, st));
  note_launch();
  k_sum_table<<<grid_elems(s->N), 256, 0, st>>>(s->table, s->G, s->gS, s->n, s->N);
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
  // the transposed copy of x is kept current by the update kernel
  (void)p;
  if (!refresh && sub < 0) return PET_ERR_ARG;
  const int b = (int)(k & 1);
  float *gk = s->gbuf[b], *gTk = s->gTbuf[b];
  pet_status e = fork_prior(s, st, b ^ 1);
  if (e != PET_OK) return e;
  const bool importance = s->o.sampling == PET_SAMPLE_IMPORTANCE;
  if (refresh) {
    if (!s->o.low_memory) {
      for (int t = 0; t < s->n; ++t) {
        float *Tt = s->table + (size_t)t * s->N;
        if (!s->o.deterministic) SCK(cudaMemsetAsync(Tt, 0, s->N * 4, st));
        e = data_grad(s, t, Tt, st, slot_of(s, k, t));
        if (e != PET_OK) return e;
      }
      note_launch();
      k_sum_table<<<ge, 256, 0, st>>>(s->table, s->G, nullptr, s->n, s->N);
      e = join_prior(s, st);
      if (e != PET_OK) return e;
      if (importance) {
        note_launch();
        k_sub_norms<<<dim3(kNormBlocks, s->n), 256, 0, st>>>(s->table, s->gS, nullptr, s->n, s->N, 1,
                                                             s->norm_part);
      }
    } else if (!importance) {
      // table-free: the full data gradient at the snapshot in one launch over all views
      SCK(cudaMemsetAsync(s->G, 0, s->N * 4, st));
      e = data_grad(s, -1, s->G, st, slot_of(s, k, 0));
      if (e != PET_OK) return e;
      e = join_prior(s, st);
      if (e != PET_OK) return e;
    } else {
      // table-free with importance sampling: each subset gradient is folded into G
      // (and cleared) by the kernel that takes its norm
      SCK(cudaMemsetAsync(s->G, 0, s->N * 4, st));
      e = join_prior(s, st);
      if (e != PET_OK) return e;
      for (int t = 0; t < s->n; ++t) {
        e = data_grad(s, t, gk, st, slot_of(s, k, t));
        if (e != PET_OK) return e;
        note_launch();
        k_sub_norms<<<dim3(kNormBlocks, 1), 256, 0, st>>>(gk, s->gS, s->G, s->n, s->N, 0,
                                                          s->norm_part + (size_t)t * kNormBlocks);
      }
    }
    if (importance) {
      note_launch();
      k_probs<<<1, 256, 0, st>>>(s->norm_part, kNormBlocks, s->n, s->prob);
      SCK(cudaMemcpyAsync(s->gSh, s->gS, s->N * 4, cudaMemcpyDeviceToDevice, st));
    }
    if (s->xhatT) SCK(cudaMemcpyAsync(s->xhatT, p->d_xT, s->N * 4, cudaMemcpyDeviceToDevice, st));
    note_launch();
    k_bb_dots<<<ge, 256, 0, st>>>(s->x, s->xhat_old, s->G, s->gS, s->Gfull_old, s->D, s->N, s->part);
    note_launch();
    k_bb_final<<<1, 256, 0, st>>>(s->part, (int)ge, s->st, s->o.bb_until <= 0 || k <= s->o.bb_until ? 1 : 0);
    note_launch();
    if (s->N >= kUpdIlpVoxels) k_update_ilp<3><<<tile_grid(s), dim3(32, 8), 0, st>>>(upd_args(s, -1, k));
    else k_update<3><<<tile_grid(s), dim3(32, 8), 0, st>>>(upd_args(s, -1, k));
  } else {
    const int *sub_dev = nullptr;
    if (importance) {
      note_launch();
      k_draw<<<1, 32, 0, st>>>(s->prob, s->n, (unsigned long long)s->o.seed, k, s->d_sub, s->d_w);
      sub_dev = s->d_sub;
    }
    e = data_grad(s, sub, gk, st, slot_of(s, k, -1), false, sub_dev, nullptr, nullptr, MODE_GRAD, gTk);
    if (e != PET_OK) return e;
    if (s->o.low_memory) {  // minus the subset gradient at the snapshot
      e = data_grad(s, sub, gk, st, -1, false, sub_dev, s->xhat_old, s->xhatT, MODE_NGRAD, gTk);
      if (e != PET_OK) return e;
    }
    if (p->res && !s->o.deterministic) {  // (P G)^T = G P^T, once on the combined accumulators
      SCK(launch_transpose(gTk, gk, p->g.nx, p->g.ny, p->g.nz, 1, 2, st));
      SCK(apply_res(p, gk, st));
    }
    e = join_prior(s, st);
    if (e != PET_OK) return e;
    UpdArgs a = upd_args(s, sub, k);
    a.g = gk;
    a.gT = gTk;
    note_launch();
    const bool ilp = s->N >= kUpdIlpVoxels;
    if (s->o.algo == PET_SGD) {
      if (ilp) k_update_ilp<0><<<tile_grid(s), dim3(32, 8), 0, st>>>(a);
      else k_update<0><<<tile_grid(s), dim3(32, 8), 0, st>>>(a);
    } else if (s->o.algo == PET_SAGA) {
      if (ilp) k_update_ilp<1><<<tile_grid(s), dim3(32, 8), 0, st>>>(a);
      else k_update<1><<<tile_grid(s), dim3(32, 8), 0, st>>>(a);
    } else {
      if (ilp) k_update_ilp<2><<<tile_grid(s), dim3(32, 8), 0, st>>>(a);
      else k_update<2><<<tile_grid(s), dim3(32, 8), 0, st>>>(a);
    }
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
  // the plan's transposed image may have been used by other calls since the last run
  SCK(to_frames(s->plan, s->x, st));
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
      s->capturing_kind = kind;
      s->kind_slots[kind].clear();
      const long long before = launch_count();
      SCK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
      pet_status ie = PET_OK;
      for (int j = 0; j < n && ie == PET_OK; ++j) ie = iterate(s, k0 + j, subs[j], s->cap_stream);
      cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &graph);
      const long long captured = launch_count() - before;  // nodes, not launches yet
      note_launch(-captured);
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
      note_launch(captured);
      for (int sl : s->kind_slots[kind]) s->pending[sl] = 1;
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

extern "C" pet_status pet_solver_profile(pet_solver *s, int enable) {
  if (!s) return PET_ERR_ARG;
  if (enable && s->ev0.empty()) {
    const int ns = n_slots(s);
    s->ev0.resize(ns);
    s->ev1.resize(ns);
    s->pending.assign(ns, 0);
    for (int i = 0; i < ns; ++i)
      if (cudaEventCreate(&s->ev0[i]) != cudaSuccess || cudaEventCreate(&s->ev1[i]) != cudaSuccess)
        return PET_ERR_CUDA;
  }
  s->profile = enable != 0;
  for (auto &e : s->exec)
    if (e) { cudaGraphExecDestroy(e); e = nullptr; }
  return PET_OK;
}

extern "C" pet_status pet_solver_kernel_time(pet_solver *s, double *total_ms, long long *launches) {
  if (!s || !total_ms || !launches) return PET_ERR_ARG;
  for (size_t i = 0; i < s->pending.size(); ++i) {
    if (!s->pending[i]) continue;
    float ms = 0.f;
    if (cudaEventSynchronize(s->ev1[i]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, s->ev0[i], s->ev1[i]) != cudaSuccess)
      return PET_ERR_CUDA;
    s->prof_ms += ms;
    s->prof_n += 1;
    s->pending[i] = 0;
  }
  *total_ms = s->prof_ms;
  *launches = s->prof_n;
  s->prof_ms = 0.0;
  s->prof_n = 0;
  return PET_OK;
}

extern "C" long long pet_launch_count(void) { return launch_count(); }

// ----------------------------------------------------------------- batches
// Many independent reconstructions (each its own plan and solver) advanced together:
// every iteration is one launch per phase for all of them (fused subset gradient, RDP
// gradient, estimator + step, accumulator clear), and iters_per_graph iterations are
// captured once into a CUDA graph that is replayed after uploading each batch epoch's
// per-instance subset and iteration indices.
struct pet_batch {
  std::vector<pet_solver *> s;
  int nj = 0, E = 8, K = 2, split = 1, algo = PET_SAGA;
  GradJob *d_gjobs = nullptr;
  RdpJob *d_rjobs = nullptr;
  UpdArgs *d_ujobs = nullptr;
  ClearJob *d_cjobs = nullptr;
  int *d_gbegin = nullptr, *d_rbegin = nullptr, *d_ubegin = nullptr, *d_cbegin = nullptr;
  int gblocks = 0, rblocks = 0, ublocks = 0, cblocks = 0;
  int *d_sub = nullptr;
  long long *d_k = nullptr;
  int *h_sub[2] = {nullptr, nullptr};
  long long *h_k[2] = {nullptr, nullptr};
  cudaEvent_t up[2] = {nullptr, nullptr};
  int buf = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  cudaStream_t side = nullptr;  // the prior's gradients, concurrent with the subset gradients
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<char> after_single;  // instance ran its last iteration alone (accumulators to clear)
  std::vector<char> solo;          // instance always runs alone (no batched form of its options)
  int rdp_zch = 0;                 // slices per batched RDP stencil block (0: each plan's own)
};

static void batch_free(pet_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  for (int i = 0; i < 2; ++i) {
    if (b->up[i]) cudaEventDestroy(b->up[i]);
    cudaFreeHost(b->h_sub[i]);
    cudaFreeHost(b->h_k[i]);
  }
  cudaFree(b->d_gjobs); cudaFree(b->d_rjobs); cudaFree(b->d_ujobs); cudaFree(b->d_cjobs);
  cudaFree(b->d_gbegin); cudaFree(b->d_rbegin); cudaFree(b->d_ubegin); cudaFree(b->d_cbegin);
  cudaFree(b->d_sub); cudaFree(b->d_k);
  delete b;
}

extern "C" void pet_batch_destroy(pet_batch *b) { batch_free(b); }

extern "C" pet_status pet_batch_create(pet_solver *const *solvers, int n, int iters_per_graph, pet_batch **out) {
  if (!solvers || !out || n < 1 || iters_per_graph < 1) return PET_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    const pet_solver *si = solvers[i];
    if (!si) return PET_ERR_ARG;
    if (si->o.algo != solvers[0]->o.algo) return PET_ERR_UNSUPPORTED;
    for (int j = 0; j < i; ++j)
      if (solvers[j]->plan == si->plan || solvers[j] == si) return PET_ERR_ARG;  // scratch is per plan
  }
  pet_batch *b = new pet_batch();
  b->s.assign(solvers, solvers + n);
  // options without a batched form run alone, one iteration at a time, inside every
  // window: TOF plans, the deterministic backprojector, the table-free SVRG, importance
  // sampling, the resolution model (the batched launches read x directly)
  b->solo.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    const pet_solver *si = solvers[i];
    b->solo[i] = si->plan->T != 1 || si->o.deterministic || si->o.low_memory ||
                 si->o.sampling == PET_SAMPLE_IMPORTANCE || si->plan->res;
  }
  b->after_single.assign(n, 1);  // the solvers may have run alone before
  b->nj = n;
  b->E = iters_per_graph;
  b->algo = solvers[0]->o.algo;
  const size_t ne = (size_t)b->E * n;
  bool ok = cudaMalloc(&b->d_gjobs, ne * sizeof(GradJob)) == cudaSuccess &&
            cudaMalloc(&b->d_rjobs, n * sizeof(RdpJob)) == cudaSuccess &&
            cudaMalloc(&b->d_ujobs, ne * sizeof(UpdArgs)) == cudaSuccess &&
            cudaMalloc(&b->d_cjobs, n * sizeof(ClearJob)) == cudaSuccess &&
            cudaMalloc(&b->d_gbegin, (n + 1) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->d_rbegin, (n + 1) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->d_ubegin, (n + 1) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->d_cbegin, (n + 1) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->d_sub, ne * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->d_k, ne * sizeof(long long)) == cudaSuccess;
  for (int i = 0; i < 2 && ok; ++i)
    ok = cudaMallocHost(&b->h_sub[i], ne * sizeof(int)) == cudaSuccess &&
         cudaMallocHost(&b->h_k[i], ne * sizeof(long long)) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->up[i], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) == cudaSuccess &&
       cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) == cudaSuccess &&
       cudaMemset(b->d_sub, 0, ne * sizeof(int)) == cudaSuccess &&
       cudaMemset(b->d_k, 0, ne * sizeof(long long)) == cudaSuccess;
  if (!ok) { batch_free(b); return PET_ERR_NOMEM; }
  *out = b;
  return PET_OK;
}

// Job tables for the current buffers of every instance (rebuilt at each run: the
// stepsize logs may have been reallocated).
static pet_status batch_tables(pet_batch *b) {
  const int n = b->nj, E = b->E;
  std::vector<GradJob> gj((size_t)E * n);
  std::vector<UpdArgs> uj((size_t)E * n);
  std::vector<RdpJob> rj(n);
  std::vector<ClearJob> cj(n);
  std::vector<int> gb(n + 1), rb(n + 1), ub(n + 1), cb(n + 1);
  gb[0] = rb[0] = ub[0] = cb[0] = 0;
  for (int i = 0; i < n; ++i) {
    pet_solver *s = b->s[i];
    pet_plan *p = s->plan;
    for (int j = 0; j < E; ++j) {
      GradJob &g = gj[(size_t)j * n + i];
      g.P = p->dp;
      g.subset_dev = b->d_sub + (size_t)j * n + i;
      g.x = s->x;
      g.xT = p->d_xT;
      g.g = s->g;
      g.gT = p->d_gT;
      UpdArgs a = upd_args(s, 0, 0);
      a.subset_dev = b->d_sub + (size_t)j * n + i;
      a.k_dev = b->d_k + (size_t)j * n + i;
      uj[(size_t)j * n + i] = a;
    }
    rj[i].a = prior_args(s, s->o.beta);
    rj[i].x = s->x;
    rj[i].grad = s->gS;
    cj[i].a = s->g;
    cj[i].b = p->d_gT;
    cj[i].N = s->N;
    if (b->rdp_zch) rj[i].a.zch = b->rdp_zch;
    const bool on = !b->solo[i];  // instances that always run alone get no batched blocks
    gb[i + 1] = gb[i] + (on ? grad_blocks_shape(p->dp, p->vs_max, b->K, b->split) : 0);
    rb[i + 1] = rb[i] + (on ? rdp_blocks(p->g.nx, p->g.ny, p->g.nz, rj[i].a.zch) : 0);
    ub[i + 1] = ub[i] + (on ? ((p->g.nx + 31) / 32) * ((p->g.ny + 31) / 32) * p->g.nz : 0);
    cb[i + 1] = cb[i] + (on ? (int)std::max<size_t>(1, std::min<size_t>(256, (s->N / 4 + 255) / 256)) : 0);
  }
  b->gblocks = gb[n];
  b->rblocks = rb[n];
  b->ublocks = ub[n];
  b->cblocks = cb[n];
  if (cudaMemcpy(b->d_gjobs, gj.data(), gj.size() * sizeof(GradJob), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_ujobs, uj.data(), uj.size() * sizeof(UpdArgs), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_rjobs, rj.data(), rj.size() * sizeof(RdpJob), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_cjobs, cj.data(), cj.size() * sizeof(ClearJob), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_gbegin, gb.data(), gb.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_rbegin, rb.data(), rb.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_ubegin, ub.data(), ub.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_cbegin, cb.data(), cb.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return PET_ERR_CUDA;
  return PET_OK;
}

// One batch iteration j of the captured epoch (all instances).
static pet_status batch_iteration(pet_batch *b, int j, cudaStream_t st) {
  const int n = b->nj;
  SCK(cudaEventRecord(b->ev_fork, st));
  SCK(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
  const int *sub = b->d_sub + (size_t)j * n;
  SCK(launch_rdp_batch(b->d_rjobs, b->d_rbegin, n, b->rblocks, sub, b->side));
  SCK(cudaEventRecord(b->ev_join, b->side));
  SCK(launch_grad_batch(b->d_gjobs + (size_t)j * n, b->d_gbegin, n, b->gblocks, b->K, b->split, st));
  SCK(cudaStreamWaitEvent(st, b->ev_join, 0));
  note_launch();
  const UpdArgs *uj = b->d_ujobs + (size_t)j * n;
  if (b->algo == PET_SAGA) k_update_batch<1><<<b->ublocks, dim3(32, 8), 0, st>>>(uj, b->d_ubegin, n);
  else if (b->algo == PET_SVRG) k_update_batch<2><<<b->ublocks, dim3(32, 8), 0, st>>>(uj, b->d_ubegin, n);
  else k_update_batch<0><<<b->ublocks, dim3(32, 8), 0, st>>>(uj, b->d_ubegin, n);
  note_launch();
  k_clear_batch<<<b->cblocks, 256, 0, st>>>(b->d_cjobs, b->d_cbegin, n, sub);
  SCK(cudaGetLastError());
  return PET_OK;
}

extern "C" pet_status pet_batch_set_grad_shape(pet_batch *b, int planes_per_thread, int parts) {
  if (!b) return PET_ERR_ARG;
  if (!(planes_per_thread == 1 || planes_per_thread == 2 || planes_per_thread == 4) ||
      !(parts == 1 || parts == 2 || parts == 4 || parts == 8))
    return PET_ERR_ARG;
  b->K = planes_per_thread;
  b->split = parts;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  return PET_OK;
}

static pet_status batch_prepare(pet_batch *b, long long niter, cudaStream_t st) {
  for (pet_solver *s : b->s) {
    pet_status e = grow_tau_log(s, s->k + niter);
    if (e != PET_OK) return e;
    SCK(to_frames(s->plan, s->x, st));
    if (!s->initialised) {
      if (s->o.algo == PET_SAGA) {
        e = saga_init(s, st);
        if (e != PET_OK) return e;
      }
      s->initialised = true;
    }
  }
  return batch_tables(b);
}

extern "C" pet_status pet_batch_autotune(pet_batch *b, void *stream, int *planes_per_thread, int *parts) {
  if (!b) return PET_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  pet_status e = batch_prepare(b, 0, st);
  if (e != PET_OK) return e;
  SCK(cudaMemsetAsync(b->d_sub, 0, (size_t)b->E * b->nj * sizeof(int), st));
  cudaEvent_t e0, e1;
  SCK(cudaEventCreate(&e0));
  SCK(cudaEventCreate(&e1));
  const int ks[3] = {1, 2, 4}, ss[4] = {1, 2, 4, 8};
  // two rounds over the shapes, 8 timed launches each after 2 untimed; each shape keeps
  // its faster round
  float tmin[3][4];
  for (auto &row : tmin)
    for (float &t : row) t = 1e30f;
  for (int round = 0; round < 2 && e == PET_OK; ++round)
    for (int a = 0; a < 3 && e == PET_OK; ++a)
      for (int c = 0; c < 4; ++c) {
        b->K = ks[a];
        b->split = ss[c];
        e = batch_tables(b);
        if (e != PET_OK) break;
        float ms = 0.f;
        for (int it = 0; it < 10; ++it) {
          if (it == 2) cudaEventRecord(e0, st);
          launch_grad_batch(b->d_gjobs, b->d_gbegin, b->nj, b->gblocks, b->K, b->split, st);
        }
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          e = PET_ERR_CUDA;
          break;
        }
        tmin[a][c] = std::min(tmin[a][c], ms);
      }
  float best = 1e30f;
  int bk = 2, bs = 1;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 4; ++c)
      if (tmin[a][c] < best) { best = tmin[a][c]; bk = ks[a]; bs = ss[c]; }
  // RDP stencil tile of the batched prior launch (slices per block, one for all instances)
  const int zs[3] = {2, 4, 8};
  float zbest = 1e30f;
  int bz = kRdpZchDefault;
  for (int round = 0; round < 2 && e == PET_OK; ++round)
    for (int zch : zs) {
      b->rdp_zch = zch;
      e = batch_tables(b);
      if (e != PET_OK) break;
      float ms = 0.f;
      for (int it = 0; it < 10; ++it) {
        if (it == 2) cudaEventRecord(e0, st);
        launch_rdp_batch(b->d_rjobs, b->d_rbegin, b->nj, b->rblocks, nullptr, st);
      }
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        e = PET_ERR_CUDA;
        break;
      }
      if (ms < zbest) { zbest = ms; bz = zch; }
    }
  b->rdp_zch = bz;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->K = bk;
  b->split = bs;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (e != PET_OK) return e;
  e = batch_tables(b);
  if (e != PET_OK) return e;
  if (b->cblocks > 0) {
    note_launch();
    k_clear_batch<<<b->cblocks, 256, 0, st>>>(b->d_cjobs, b->d_cbegin, b->nj, nullptr);  // discard the trial gradients
  }
  SCK(cudaGetLastError());
  SCK(cudaStreamSynchronize(st));
  if (planes_per_thread) *planes_per_thread = bk;
  if (parts) *parts = bs;
  return PET_OK;
}

// An iteration in [k0, k0 + len) that the batched phases cannot run for this solver: a
// preconditioner update or an SVRG snapshot refresh (n subset gradients and a step).
static bool window_has_event(const pet_solver *s, long long k0, long long len) {
  if (epoch_has_pc(s, k0, len)) return true;
  if (s->o.algo != PET_SVRG) return false;
  const long long period = (long long)s->o.omega * s->n;
  const long long next = ((k0 + period - 1) / period) * period;  // first refresh at or after k0
  return next < k0 + len;
}

extern "C" pet_status pet_batch_run(pet_batch *b, long long niter, void *stream) {
  if (!b || niter < 0) return PET_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  for (pet_solver *s : b->s)
    if (!s->order.empty() && s->k + niter > (long long)s->order.size()) return PET_ERR_ARG;
  pet_status e = batch_prepare(b, niter, st);
  if (e != PET_OK) return e;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  const int n = b->nj, E = b->E;
  long long done = 0;
  std::vector<char> alone(n);
  while (done < niter) {
    // An instance whose window holds an event (or a final window shorter than E) runs the
    // window alone, iteration by iteration; the others run the captured batched window,
    // in which the lone instances are marked kBatchSkip.
    const long long len = std::min<long long>(E, niter - done);
    int nalone = 0;
    for (int i = 0; i < n; ++i) {
      alone[i] = b->solo[i] || len < E || window_has_event(b->s[i], b->s[i]->k, E);
      nalone += alone[i];
    }
    for (int i = 0; i < n; ++i) {
      if (!alone[i]) continue;
      pet_solver *s = b->s[i];
      for (long long j = 0; j < len; ++j) {
        e = iterate(s, s->k, subset_of(s, s->k), st);
        if (e != PET_OK) return e;
        s->k += 1;
      }
      b->after_single[i] = 1;
    }
    done += len;
    if (nalone == n) continue;
    // A single-solver iteration leaves its accumulator pair for the next one to clear;
    // the batched phases use (g, the plan's transposed accumulator), so clear it here
    // (after single-solver iterations only: a batched window leaves both clean).
    for (int i = 0; i < n; ++i) {
      pet_solver *s = b->s[i];
      if (alone[i] || !b->after_single[i]) continue;
      if (s->k > 0) {
        const int pb = (int)((s->k - 1) & 1);
        note_launch();
        k_clear2<<<grid_elems(s->N / 4), 256, 0, st>>>(s->gbuf[pb], s->gTbuf[pb], s->N);
      }
      b->after_single[i] = 0;
    }
    SCK(cudaGetLastError());
    if (!b->exec) {
      cudaGraph_t graph = nullptr;
      const long long before = launch_count();
      SCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
      pet_status ie = PET_OK;
      for (int j = 0; j < E && ie == PET_OK; ++j) ie = batch_iteration(b, j, b->cap);
      const cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
      note_launch(-(launch_count() - before));
      if (ie != PET_OK) { if (graph) cudaGraphDestroy(graph); return ie; }
      if (ce != cudaSuccess) return PET_ERR_CUDA;
      const cudaError_t ie2 = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie2 != cudaSuccess) return PET_ERR_CUDA;
    }
    const int bb = b->buf;
    b->buf ^= 1;
    SCK(cudaEventSynchronize(b->up[bb]));  // the previous upload from this host buffer is done
    for (int j = 0; j < E; ++j)
      for (int i = 0; i < n; ++i) {
        pet_solver *s = b->s[i];
        b->h_sub[bb][(size_t)j * n + i] = alone[i] ? kBatchSkip : subset_of(s, s->k + j);
        b->h_k[bb][(size_t)j * n + i] = s->k + j;
      }
    SCK(cudaMemcpyAsync(b->d_sub, b->h_sub[bb], (size_t)E * n * sizeof(int), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(b->d_k, b->h_k[bb], (size_t)E * n * sizeof(long long), cudaMemcpyHostToDevice, st));
    SCK(cudaEventRecord(b->up[bb], st));
    SCK(cudaGraphLaunch(b->exec, st));
    note_launch(4LL * E);
    for (int i = 0; i < n; ++i)
      if (!alone[i]) b->s[i]->k += E;
  }
  return PET_OK;
}
