// Fused TOF subset gradient (eq. 5 with the KL data term of Sec. 1.2 and the TOF-weighted
// Joseph projector) for sm_103a, built around a sliding window of TOF bins.
//
// A sample at position t along its LOR meets the bins b with |t - c_b| < R = 3 sigma + w/2
// (the truncated-Gaussian weight of bin b is F(t - c_b), F even, zero beyond R), at most
// WIN consecutive bins.  Along a LOR t moves monotonically, so each thread keeps the
// WIN bins around its current sample in registers and retires the lowest bin when the
// window moves past it (forward: its finished sum goes to shared memory; backward: the
// next bin's q enters the window).  LORs whose t decreases along the driving axis are
// traversed with t' = -t and mirrored bins b' = T-1-b (F is even and c_{T-1-b} = -c_b),
// so every window slides upward.
//
// Weights: F is tabulated at the spacing h = w/M (M = 1024 per bin width) and
// interpolated linearly.  With x = (t - c_0 + R)/h the node index of bin b is
// floor(x) - b M, so every bin of the window shares the fraction of x and the table can
// be stored by rows: row ridx holds, for each pair of window bins (j, j+1), the values
// (F(n_j), F(n_{j+1})) and slopes (F(n_j + 1) - F(n_j), ...) at their nodes n_j, and
// one sample reads one row.  The interpolation error is below h^2/8 max|F''| ~ 1e-7
// (and h/4 times the slope jump, ~1.4e-6 absolute, at the four kinks of the truncation,
// where F is ~1e-2 of its peak).  Pairs of bins are evaluated with the packed FP32x2
// FMA of sm_100+ (two independent round-to-nearest FMAs, the same results as two FFMAs).
//
// Planes per thread (K = 2 or 4): LORs of one view and radial bin on consecutive planes
// of equal axial slope (plane groups built on the host) share their in-plane sample
// positions and their positions t along the LOR, hence the TOF weights of every sample.
//
// Parts (SPLIT): the driving planes of a LOR are interleaved over SPLIT threads; each
// keeps its own window; the bin sums are combined in a fixed order with compensation.
// With one part a thread owns its LORs from the forward sums to the backprojection, so
// no block barrier separates the phases.
#include <algorithm>
#include <climits>

#include "packed_f32x2.cuh"
#include "pet_internal.cuh"

namespace petgb {

namespace {

__device__ __forceinline__ void kahan(float &sum, float &c, float v) {
  const float yk = v - c;
  const float tk = sum + yk;
  c = (tk - sum) - yk;
  sum = tk;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < NT / 32 ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// Window coordinate of sample i: x' = xs0 + i dxs; u = floor(x') split into the window's
// lowest bin (u >> log2 M) and the table row (u & (M-1)); f the shared fraction.  u is
// clamped so that a window never starts more than 4 bins below 0 or beyond T + WIN + 4.
struct WinPos {
  int kb, row;
  float f;
};

__device__ __forceinline__ WinPos win_pos(float xs, int umax) {
  const float fu = floorf(xs);
  int u = (int)fu;
  u = min(max(u, -4 * kTofM), umax);
  WinPos w;
  w.kb = u >> kTofLogM;
  w.row = u & (kTofM - 1);
  w.f = xs - fu;
  return w;
}

// Weights of the WIN window bins as WIN/2 pairs: w2[p] = (w_{2p}, w_{2p+1}).
template <int WIN>
__device__ __forceinline__ void win_weights(const float4 *__restrict__ tab, int row, float f, float2 (&w2)[WIN / 2]) {
  const float4 *r = tab + row * (WIN / 2);
  const float2 ff = make_float2(f, f);
#pragma unroll
  for (int p = 0; p < WIN / 2; ++p) {
    const float4 e = r[p];  // (F_2p, F_2p+1, slope_2p, slope_2p+1)
    w2[p] = fma2(ff, make_float2(e.z, e.w), make_float2(e.x, e.y));
  }
}

}  // namespace

// One LOR group (K planes of one view and radial bin; part `part` of SPLIT) from the forward
// TOF sums to the backprojection; returns this thread's share of the KL value.  s_acc is
// the block's bin array (column tid of each row belongs to this thread; with SPLIT > 1 the
// parts of LOR group tl exchange sums through columns j LPB + tl, so every thread of the
// block must call this together).  The caller has cleared this thread's column.
// ZI: the planes of every group lie a whole number of slices apart (checked on the host),
// so they share the fraction of their axial position along the LOR: plane k samples row
// floor(z_0) + dz_k with the weight of plane 0, one floor per sample instead of K.
template <int K, int WIN, int SPLIT, int NT, bool ZI = false>
__device__ __forceinline__ double tof_group(const DevPlan &P, const float4 *__restrict__ s_tab, float *s_acc,
                                            int v, int r, int grp, bool ok, int part, int tl, int tid,
                                            const float *__restrict__ x, const float *__restrict__ xT,
                                            float *__restrict__ g, float *__restrict__ gT, int mode, bool want_kl) {
  constexpr int LPB = NT / SPLIT;
  constexpr int WP = WIN / 2;
  const int T = P.T;
  // shared in-plane geometry and the planes of the group
  const float4 vw = __ldg(&P.view[v]);
  const float4 vr = __ldg(&P.vr[v * P.nrad + r]);
  const bool xdrive = vw.x != 0.f;
  const float dfb = vw.y, dau = vw.z, fb0 = vr.x, t0b = vr.y, inv2h = vr.z;
  const float g1 = dau * inv2h, g2 = t0b * inv2h;
  const int Na = xdrive ? P.nx : P.ny;
  const int Nb = xdrive ? P.ny : P.nx;
  int pk[K];
  bool pv[K];
  float fz0[K], dfz[K];
  int dzk[K];  // ZI: slice offset of plane k from plane 0
  float zs0 = 0.f;
  float sec = 1.f;
  float lo_b = 0.f, hi_b = (float)(Na - 1);
  clip_range(fb0, dfb, -1.f, (float)Nb, lo_b, hi_b);
  float lo = 1e30f, hi = -1e30f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int p = K == 1 ? grp : __ldg(&(K == 2 ? P.tof_grp2 : P.tof_grp4)[K * grp + k]);
    pv[k] = ok && p >= 0;
    pk[k] = pv[k] ? p : 0;
    const float4 pl = __ldg(&P.plane[pk[k]]);
    dfz[k] = g1 * pl.y;
    fz0[k] = fmaf(g2, pl.y, pl.x);
    if (k == 0) {  // planes of a group share their axial slope, hence sec and t
      const float kk = pl.z * inv2h;
      sec = sqrtf(fmaf(kk, kk, 1.f));
      zs0 = pl.x;
    }
    dzk[k] = k == 0 ? 0 : __float2int_rn(pl.x - zs0);
    float lk = lo_b, hk = hi_b;
    clip_range(fz0[k], dfz[k], -1.f, (float)P.nz, lk, hk);
    if (pv[k] && lk <= hk) { lo = fminf(lo, lk); hi = fmaxf(hi, hk); }
  }
  Lor L = {};
  if (lo <= hi) {
    lo = fmaxf(lo, -2.f);
    hi = fminf(hi, (float)Na + 1.f);
    L.i0 = max(0, (int)floorf(lo) - 1);
    L.i1 = min(Na - 1, (int)ceilf(hi) + 1);
  } else {
    L.i0 = 1;
    L.i1 = 0;
  }
  warp_uniform_range(L, ok);
  // the forward gathers from the zero-padded copy of the image in this view's frame
  // (2 voxels of zeros on both sides of the b and z axes): indices clamped to the padding
  // need no bounds tests, and samples outside the image read zeros
  const float *imgp = xdrive ? P.tof_xtp : P.tof_xp;
  const int Nbp = Nb + 2 * kTofPad;
  const int planep = Na * Nbp;
  // window coordinate along the (possibly mirrored) LOR
  const bool mirror = dau < 0.f;
  const float sg = mirror ? -1.f : 1.f;
  const float xs0 = fmaf(sg * t0b * sec, P.tofw_inv_h, P.tofw_off);
  const float dxs = sg * dau * sec * P.tofw_inv_h;
  const int umax = (T + WIN + 4) * kTofM;
  if (mode != MODE_SENS) {
    float2 acc[K][WP];  // bins (2p, 2p+1) of the window for each plane
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int q = 0; q < WP; ++q) acc[k][q] = make_float2(0.f, 0.f);
    int kbase = INT_MIN;
    for (int i = L.i0 + part; i <= L.i1; i += SPLIT) {
      if (!ok || i >= Na) continue;
      const float fb = fmaf((float)i, dfb, fb0);
      const float fbf = floorf(fb);
      const int ib = min(max((int)fbf, -kTofPad), Nb);
      const float wb = fb - fbf;
      const int rowp = i * Nbp + ib + kTofPad;
      // bilinear interpolation: the two rows of each plane in one packed pair, then the
      // axial step for two planes at a time
      const float2 wbb = make_float2(wb, wb), wbb1 = make_float2(1.f - wb, 1.f - wb);
      float2 h[K];
      float wzk[K];
      int iz0 = 0;
      float wz0 = 0.f;
      if (ZI) {
        const float fz = fmaf((float)i, dfz[0], fz0[0]);
        const float fzf = floorf(fz);
        iz0 = (int)fzf;
        wz0 = fz - fzf;
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        int izk;
        if (ZI) {
          izk = iz0 + dzk[k];
          wzk[k] = wz0;
        } else {
          const float fz = fmaf((float)i, dfz[k], fz0[k]);
          const float fzf = floorf(fz);
          izk = (int)fzf;
          wzk[k] = fz - fzf;
        }
        const int iz = min(max(izk, -kTofPad), P.nz);
        const int base = (iz + kTofPad) * planep + rowp;
        const float v00 = __ldg(imgp + base);
        const float v01 = __ldg(imgp + base + 1);
        const float v10 = __ldg(imgp + base + planep);
        const float v11 = __ldg(imgp + base + planep + 1);
        h[k] = fma2(wbb, make_float2(v01, v11), mul2(wbb1, make_float2(v00, v10)));
      }
      float val[K];
      if (K == 1) {
        val[0] = fmaf(wzk[0], h[0].y, (1.f - wzk[0]) * h[0].x);
      } else {
#pragma unroll
        for (int k = 0; k + 1 < K; k += 2) {
          const float2 wz2 = make_float2(wzk[k], wzk[k + 1]);
          const float2 r2 = fma2(wz2, make_float2(h[k].y, h[k + 1].y),
                                 mul2(sub2(make_float2(1.f, 1.f), wz2), make_float2(h[k].x, h[k + 1].x)));
          val[k] = r2.x;
          val[k + 1] = r2.y;
        }
      }
      bool any = false;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        val[k] = pv[k] ? val[k] : 0.f;
        any |= val[k] != 0.f;
      }
      if (!any) continue;
      const WinPos wp = win_pos(fmaf((float)i, dxs, xs0), umax);
      if (kbase == INT_MIN) kbase = wp.kb;
      while (kbase < wp.kb) {  // retire the lowest bin of the window, shift the rest down
        const int b = mirror ? T - 1 - kbase : kbase;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if ((unsigned)kbase < (unsigned)T) s_acc[(k * T + b) * NT + tid] = acc[k][0].x;
#pragma unroll
          for (int q = 0; q < WP; ++q) {
            acc[k][q].x = acc[k][q].y;
            acc[k][q].y = q + 1 < WP ? acc[k][q + 1].x : 0.f;
          }
        }
        ++kbase;
      }
      float2 w2[WP];
      win_weights<WIN>(s_tab, wp.row, wp.f, w2);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float2 vv = make_float2(val[k], val[k]);
#pragma unroll
        for (int q = 0; q < WP; ++q) acc[k][q] = fma2(vv, w2[q], acc[k][q]);
      }
    }
    if (kbase != INT_MIN) {
#pragma unroll
      for (int j = 0; j < WIN; ++j) {
        const int kb = kbase + j;
        if ((unsigned)kb < (unsigned)T) {
          const int b = mirror ? T - 1 - kb : kb;
#pragma unroll
          for (int k = 0; k < K; ++k) s_acc[(k * T + b) * NT + tid] = (j & 1) ? acc[k][j / 2].y : acc[k][j / 2].x;
        }
      }
    }
  }
  if (SPLIT > 1) __syncthreads();  // every part's bin sums are in shared memory

  // KL ratio: part p handles the bins b = p, p + SPLIT, ... of its LOR group; the parts'
  // sums are added in a fixed order with compensation; q replaces the sum of part 0.
  double kl = 0.0;
  bool anyq = false;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!pv[k]) continue;
    const size_t lor = ((size_t)v * P.nplane + pk[k]) * P.nrad + r;
    const float mL = __ldg(&P.m[lor]) * fabsf(dau) * sec;
    for (int b = part; b < T; b += SPLIT) {
      float *cell = s_acc + (k * T + b) * NT;
      float q;
      if (mode == MODE_SENS) {
        q = mL;
      } else {
        float sum = cell[tl], c = 0.f;
#pragma unroll
        for (int j = 1; j < SPLIT; ++j) kahan(sum, c, cell[j * LPB + tl]);
        const size_t bi = lor * T + b;
        const float ybar = fmaf(mL, sum, __ldg(&P.r[bi]));
        const float yb = load_y(P, bi);
        if (!(ybar > 0.f)) {
          if (yb > 0.f) atomicOr(P.err, 1);
          q = (grad_like(mode) && yb == 0.f) ? mL : 0.f;
          if (want_kl && yb == 0.f) kl += (double)fmaxf(ybar, 0.f);
        } else {
          q = grad_like(mode) ? mL * (1.f - yb / ybar) : (mode == MODE_EM ? mL * (yb / ybar) : 0.f);
          if (want_kl) {
            const double db = ybar, dy = yb;
            kl += (yb > 0.f) ? (db - dy + dy * log(dy / db)) : db;
          }
        }
        if (mode == MODE_NGRAD) q = -q;
      }
      cell[tl] = q;
      anyq |= q != 0.f;
    }
  }
  if (SPLIT > 1) {
    __syncthreads();  // every q of the block is in place
    anyq = false;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (pv[k])
        for (int b = 0; b < T; ++b) anyq |= s_acc[(k * T + b) * NT + tl] != 0.f;
  }

  if (mode != MODE_OBJ) {
    // the scatter goes to zero-padded accumulators in the view's frame (neighbours outside
    // the image land in the padding, which the combine pass after the kernel discards)
    float *outp = xdrive ? P.tof_gtp : P.tof_gp;
    float2 qw[K][WP];
    int kbase = INT_MIN;
    for (int i = L.i0 + part; i <= L.i1; i += SPLIT) {
      if (!anyq || i >= Na) continue;
      const WinPos wp = win_pos(fmaf((float)i, dxs, xs0), umax);
      if (kbase == INT_MIN || kbase < wp.kb) {
        kbase = wp.kb;  // (re)load the window's ratios; the window only moves upward
#pragma unroll
        for (int j = 0; j < WIN; ++j) {
          const int kb = kbase + j;
          const bool in = (unsigned)kb < (unsigned)T;
          const int b = mirror ? T - 1 - kb : kb;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const float qv = in ? s_acc[(k * T + b) * NT + tl] : 0.f;
            if (j & 1) qw[k][j / 2].y = qv;
            else qw[k][j / 2].x = qv;
          }
        }
      }
      float2 w2[WP];
      win_weights<WIN>(s_tab, wp.row, wp.f, w2);
      float val[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < WP; ++q) a = fma2(qw[k][q], w2[q], a);
        val[k] = a.x + a.y;
      }
      const float fb = fmaf((float)i, dfb, fb0);
      const float fbf = floorf(fb);
      const int ib = (int)fbf;
      const float wb = fb - fbf;
      if ((unsigned)(ib + 1) > (unsigned)Nb) continue;  // both in-plane neighbours outside
      const int rowp = i * Nbp + ib + kTofPad;
      const float2 wbp = make_float2(1.f - wb, wb);
      int iz0 = 0;
      float wz0 = 0.f;
      if (ZI) {
        const float fz = fmaf((float)i, dfz[0], fz0[0]);
        const float fzf = floorf(fz);
        iz0 = (int)fzf;
        wz0 = fz - fzf;
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (val[k] == 0.f) continue;
        int iz;
        float wz;
        if (ZI) {
          iz = iz0 + dzk[k];
          wz = wz0;
        } else {
          const float fz = fmaf((float)i, dfz[k], fz0[k]);
          const float fzf = floorf(fz);
          iz = (int)fzf;
          wz = fz - fzf;
        }
        if ((unsigned)(iz + 1) > (unsigned)P.nz) continue;  // both axial neighbours outside
        const int base = (iz + kTofPad) * planep + rowp;
        const float2 a = mul2(make_float2(1.f - wz, wz), make_float2(val[k], val[k]));
        const float2 lo2 = mul2(wbp, make_float2(a.x, a.x));
        atomicAdd(outp + base, lo2.x);
        atomicAdd(outp + base + 1, lo2.y);
        if (wz != 0.f) {  // the upper row of a plane through slice centres has weight 0
          const float2 up2 = mul2(wbp, make_float2(a.y, a.y));
          atomicAdd(outp + base + planep, up2.x);
          atomicAdd(outp + base + planep + 1, up2.y);
        }
      }
    }
  }
  return kl;
}

// Fused TOF gradient: forward (windowed TOF sums), KL ratio, backprojection.  NT threads
// per block, one LOR group per thread (or part); dynamic shared memory: the weight table
// (kTofM rows of WIN/2 float4) then the bin sums / ratios s_acc[(k T + b) NT + tid].
template <int K, int WIN, int SPLIT, int NT>
__global__ void __launch_bounds__(NT, 2) k_grad_tofk(DevPlan P, int subset, const int *subset_dev,
                                                     const float *__restrict__ x, const float *__restrict__ xT,
                                                     float *__restrict__ g, float *__restrict__ gT,
                                                     double *__restrict__ kl_part, int mode) {
  constexpr int LPB = NT / SPLIT;  // LOR groups per block
  extern __shared__ float4 s_dyn[];
  float4 *s_tab = s_dyn;
  float *s_acc = reinterpret_cast<float *>(s_dyn + kTofM * (WIN / 2));
  const int tid = threadIdx.x;
  for (int k = tid; k < kTofM * (WIN / 2); k += NT) s_tab[k] = __ldg(&P.tofw_tab[k]);
  for (int k = 0; k < K * P.T; ++k) s_acc[k * NT + tid] = 0.f;
  if (subset_dev) subset = *subset_dev;
  const int part = tid / LPB;
  const int tl = tid % LPB;
  const int nsub = subset < 0 ? 1 : P.nsub;
  const int s0 = subset < 0 ? 0 : subset;
  const int nv = (P.nview - s0 + nsub - 1) / nsub;
  const int ngrp = K == 1 ? P.nplane : (K == 2 ? P.tof_ngrp2 : P.tof_ngrp4);
  const long long uid = (long long)blockIdx.x * LPB + tl;
  const bool ok = uid < (long long)nv * ngrp * P.nrad;
  int v = 0, r = 0, grp = 0;
  if (ok) {
    r = (int)(uid % P.nrad);
    const long long t = uid / P.nrad;
    grp = (int)(t % ngrp);
    v = s0 + (int)(t / ngrp) * nsub;
  }
  __syncthreads();  // table and cleared sums ready
  const double kl = tof_group<K, WIN, SPLIT, NT>(P, s_tab, s_acc, v, r, grp, ok, part, tl, tid, x, xT, g, gT, mode,
                                                 kl_part != nullptr);
  if (kl_part) {
    const double s = block_sum<NT>(kl);
    if (tid == 0) kl_part[blockIdx.x] = s;
  }
}

// Persistent form with one part per LOR: a few blocks per SM load the table once, and each
// warp takes work units (32 consecutive radial bins of one view and plane group) from a
// counter in device memory (cleared before the launch) until none is left, so that no SM
// idles while a block waits for its slowest warp.
template <int K, int WIN, int NT, bool ZI>
__global__ void __launch_bounds__(NT, 2) k_grad_tofp(DevPlan P, int subset, const int *subset_dev,
                                                     const float *__restrict__ x, const float *__restrict__ xT,
                                                     float *__restrict__ g, float *__restrict__ gT,
                                                     double *__restrict__ kl_part, int mode) {
  extern __shared__ float4 s_dyn[];
  float4 *s_tab = s_dyn;
  float *s_acc = reinterpret_cast<float *>(s_dyn + kTofM * (WIN / 2));
  const int tid = threadIdx.x, lane = tid & 31;
  for (int k = tid; k < kTofM * (WIN / 2); k += NT) s_tab[k] = __ldg(&P.tofw_tab[k]);
  if (subset_dev) subset = *subset_dev;
  const int nsub = subset < 0 ? 1 : P.nsub;
  const int s0 = subset < 0 ? 0 : subset;
  const int nv = (P.nview - s0 + nsub - 1) / nsub;
  const int ngrp = K == 1 ? P.nplane : (K == 2 ? P.tof_ngrp2 : P.tof_ngrp4);
  const int nchunk = (P.nrad + 31) / 32;
  const long long units = (long long)nv * ngrp * nchunk;
  // per-thread KL sums live in shared memory, not in registers across the unit loop
  __shared__ double s_kl[NT];
  s_kl[tid] = 0.0;
  __syncthreads();  // table ready
  for (;;) {
    long long u = 0;
    if (lane == 0) u = atomicAdd(reinterpret_cast<unsigned long long *>(P.tof_work), 1ULL);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= units) break;  // warp-uniform
    const int chunk = (int)(u % nchunk);
    const long long t = u / nchunk;
    const int grp = (int)(t % ngrp);
    const int v = s0 + (int)(t / ngrp) * nsub;
    const int r = chunk * 32 + lane;
    const bool ok = r < P.nrad;
    for (int k = 0; k < K * P.T; ++k) s_acc[k * NT + tid] = 0.f;
    const double kl = tof_group<K, WIN, 1, NT, ZI>(P, s_tab, s_acc, v, ok ? r : 0, grp, ok, 0, tid, tid, x, xT, g, gT,
                                               mode, kl_part != nullptr);
    if (kl_part) s_kl[tid] += kl;
  }
  if (kl_part) {
    const double s = block_sum<NT>(s_kl[tid]);
    if (tid == 0) kl_part[blockIdx.x] = s;
  }
}

// Threads per block: 512 for 1 or 2 planes per thread, 256 for 4 (more registers).
template <int K>
constexpr int tofk_nt() { return K == 4 ? 256 : kTofBlock; }

bool tofk_supported(const DevPlan &P, int K) {
  if (P.T <= 1 || P.T > kTofMaxBins || !P.tofw_tab) return false;
  if (P.tofw_win < 1 || P.tofw_win > 8) return false;
  return K == 1 || (K == 2 && P.tof_grp2) || (K == 4 && P.tof_grp4);
}

int tofk_blocks(const DevPlan &P, int nv, int K, int split) {
  const long long ngrp = K == 1 ? P.nplane : (K == 2 ? P.tof_ngrp2 : P.tof_ngrp4);
  const int nt = K == 4 ? tofk_nt<4>() : kTofBlock;
  if (split == 1) {  // persistent: two blocks per SM, or fewer when there is less work
    const long long units = (long long)nv * ngrp * ((P.nrad + 31) / 32);
    const long long need = (units + nt / 32 - 1) / (nt / 32);
    return (int)std::min<long long>(need, 2LL * P.nsm);
  }
  const long long units = (long long)nv * ngrp * P.nrad;
  const int lpb = nt / split;
  return (int)((units + lpb - 1) / lpb);
}

template <int K, int WIN, int SPLIT>
static cudaError_t launch_tofk_t(const DevPlan &P, unsigned grid, int subset, const int *subset_dev, const float *x,
                                 const float *xT, float *g, float *gT, double *kl_part, int mode, cudaStream_t st) {
  constexpr int NT = tofk_nt<K>();
  const size_t smem = (size_t)kTofM * (WIN / 2) * sizeof(float4) + (size_t)K * P.T * NT * sizeof(float);
  if (SPLIT == 1) {
    cudaError_t e = cudaMemsetAsync(P.tof_work, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (K > 1 && P.tof_zint)
      k_grad_tofp<K, WIN, NT, true><<<grid, NT, smem, st>>>(P, subset, subset_dev, x, xT, g, gT, kl_part, mode);
    else
      k_grad_tofp<K, WIN, NT, false><<<grid, NT, smem, st>>>(P, subset, subset_dev, x, xT, g, gT, kl_part, mode);
  } else {
    k_grad_tofk<K, WIN, SPLIT, NT><<<grid, NT, smem, st>>>(P, subset, subset_dev, x, xT, g, gT, kl_part, mode);
  }
  return cudaGetLastError();
}

// Raises the dynamic shared-memory limit of one kernel instance to what its largest
// launch needs (the table plus K x 16 bins of sums per thread).
template <int K, int WIN, int SPLIT>
static cudaError_t tofk_attr() {
  constexpr int NT = tofk_nt<K>();
  const int bytes = (int)(kTofM * (WIN / 2) * sizeof(float4) + K * kTofMaxBins * NT * sizeof(float));
  if (SPLIT == 1) {
    cudaError_t e = cudaFuncSetAttribute(k_grad_tofp<K, WIN, NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         bytes);
    if (e == cudaSuccess && K > 1)
      e = cudaFuncSetAttribute(k_grad_tofp<K, WIN, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
  }
  return cudaFuncSetAttribute(k_grad_tofk<K, WIN, SPLIT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int K, int WIN>
static cudaError_t tofk_attr_w() {
  cudaError_t e = tofk_attr<K, WIN, 1>();
  if (e == cudaSuccess) e = tofk_attr<K, WIN, 2>();
  if (e == cudaSuccess) e = tofk_attr<K, WIN, 4>();
  if (e == cudaSuccess) e = tofk_attr<K, WIN, 8>();
  return e;
}

cudaError_t tofk_init_device() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = tofk_attr_w<1, 4>();
  if (e == cudaSuccess) e = tofk_attr_w<1, 6>();
  if (e == cudaSuccess) e = tofk_attr_w<1, 8>();
  if (e == cudaSuccess) e = tofk_attr_w<2, 4>();
  if (e == cudaSuccess) e = tofk_attr_w<2, 6>();
  if (e == cudaSuccess) e = tofk_attr_w<2, 8>();
  if (e == cudaSuccess) e = tofk_attr_w<4, 4>();
  if (e == cudaSuccess) e = tofk_attr_w<4, 6>();
  if (e == cudaSuccess) e = tofk_attr_w<4, 8>();
  return e;
}

template <int K, int WIN>
static cudaError_t launch_tofk_w(const DevPlan &P, unsigned grid, int split, int subset, const int *subset_dev,
                                 const float *x, const float *xT, float *g, float *gT, double *kl_part, int mode,
                                 cudaStream_t st) {
  switch (split) {
    case 1: return launch_tofk_t<K, WIN, 1>(P, grid, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
    case 2: return launch_tofk_t<K, WIN, 2>(P, grid, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
    case 4: return launch_tofk_t<K, WIN, 4>(P, grid, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
    default: return launch_tofk_t<K, WIN, 8>(P, grid, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
  }
}

template <int K>
static cudaError_t launch_tofk_k(const DevPlan &P, unsigned grid, int split, int subset, const int *subset_dev,
                                 const float *x, const float *xT, float *g, float *gT, double *kl_part, int mode,
                                 cudaStream_t st) {
  const int win = P.tofw_win <= 4 ? 4 : (P.tofw_win <= 6 ? 6 : 8);
  if (win == 4) return launch_tofk_w<K, 4>(P, grid, split, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
  if (win == 6) return launch_tofk_w<K, 6>(P, grid, split, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
  return launch_tofk_w<K, 8>(P, grid, split, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
}

// Zero-padded copies of the image in both view frames: xp [nz+2p][ny][nx+2p] (views
// driven along y) and xtp [nz+2p][nx][ny+2p] (views driven along x), p = kTofPad.  Only
// the interior is written; the padding was cleared when the plan was created.  One
// 32x32 tile of one slice per block, transposed through shared memory.
__global__ void __launch_bounds__(256) k_pad_frames(const float *__restrict__ x, float *__restrict__ xp,
                                                    float *__restrict__ xtp, int nx, int ny) {
  __shared__ float tile[32][33];
  const int z = blockIdx.z, x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const size_t sl = (size_t)z * nx * ny;
  const size_t slp = (size_t)(z + kTofPad) * ny * (nx + 2 * kTofPad);
  const size_t sltp = (size_t)(z + kTofPad) * nx * (ny + 2 * kTofPad);
  for (int j = ty; j < 32; j += 8) {
    const int xx = x0 + tx, yy = y0 + j;
    if (xx < nx && yy < ny) {
      const float v = x[sl + (size_t)yy * nx + xx];
      xp[slp + (size_t)yy * (nx + 2 * kTofPad) + xx + kTofPad] = v;
      tile[j][tx] = v;
    }
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int xx = x0 + j, yy = y0 + tx;
    if (xx < nx && yy < ny) xtp[sltp + (size_t)xx * (ny + 2 * kTofPad) + yy + kTofPad] = tile[tx][j];
  }
}

static cudaError_t launch_grad_tofk_core(const DevPlan &P, int K, int split, unsigned grid, int subset,
                                         const int *subset_dev, const float *x, const float *xT, float *g, float *gT,
                                         double *kl_part, int mode, cudaStream_t st);

// g += the interiors of the padded accumulators (gtp transposed back through shared
// memory); the caller then clears both padded arrays, padding included.
__global__ void __launch_bounds__(256) k_unpad_add(const float *__restrict__ gp, const float *__restrict__ gtp,
                                                   float *__restrict__ g, int nx, int ny) {
  __shared__ float tile[32][33];
  const int z = blockIdx.z, x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const size_t sl = (size_t)z * nx * ny;
  const size_t slp = (size_t)(z + kTofPad) * ny * (nx + 2 * kTofPad);
  const size_t sltp = (size_t)(z + kTofPad) * nx * (ny + 2 * kTofPad);
  for (int j = ty; j < 32; j += 8) {
    const int xx = x0 + j, yy = y0 + tx;
    if (xx < nx && yy < ny) tile[j][tx] = gtp[sltp + (size_t)xx * (ny + 2 * kTofPad) + yy + kTofPad];
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int xx = x0 + tx, yy = y0 + j;
    if (xx < nx && yy < ny) {
      const size_t i = sl + (size_t)yy * nx + xx;
      g[i] += gp[slp + (size_t)yy * (nx + 2 * kTofPad) + xx + kTofPad] + tile[tx][j];
    }
  }
}

cudaError_t launch_grad_tofk(const DevPlan &P, int K, int split, unsigned grid, int subset, const int *subset_dev,
                             const float *x, const float *xT, float *g, float *gT, double *kl_part, int mode,
                             cudaStream_t st) {
  cudaError_t e = launch_grad_tofk_core(P, K, split, grid, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
  if (e != cudaSuccess || mode == MODE_OBJ) return e;
  const dim3 tiles((P.nx + 31) / 32, (P.ny + 31) / 32, P.nz);
  note_launch();
  k_unpad_add<<<tiles, dim3(32, 8), 0, st>>>(P.tof_gp, P.tof_gtp, g, P.nx, P.ny);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t np = (size_t)(P.nz + 2 * kTofPad) * P.ny * (P.nx + 2 * kTofPad);
  const size_t ntp = (size_t)(P.nz + 2 * kTofPad) * P.nx * (P.ny + 2 * kTofPad);
  e = cudaMemsetAsync(P.tof_gp, 0, np * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.tof_gtp, 0, ntp * sizeof(float), st);
  return e;
}

static cudaError_t launch_grad_tofk_core(const DevPlan &P, int K, int split, unsigned grid, int subset,
                                         const int *subset_dev, const float *x, const float *xT, float *g, float *gT,
                                         double *kl_part, int mode, cudaStream_t st) {
  if (mode != MODE_SENS) {
    note_launch();
    k_pad_frames<<<dim3((P.nx + 31) / 32, (P.ny + 31) / 32, P.nz), dim3(32, 8), 0, st>>>(x, P.tof_xp, P.tof_xtp,
                                                                                         P.nx, P.ny);
  }
  note_launch();
  if (K == 4) return launch_tofk_k<4>(P, grid, split, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
  if (K == 2) return launch_tofk_k<2>(P, grid, split, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
  return launch_tofk_k<1>(P, grid, split, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
}

}  // namespace petgb
