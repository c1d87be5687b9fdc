// Joseph ray-driven projector kernels for sm_103a: forward projection, matched
// ray-driven backprojection, the fused subset gradient (forward -> KL ratio -> back,
// eq. 5 with the KL data term of Sec. 1.2) and the setup kernels (attenuation factors,
// sensitivity).  One thread owns one LOR; adjacent threads own adjacent radial bins of
// the same view and plane, so their samples at a given plane touch adjacent voxels of
// the driving-frame image.
#include <algorithm>
#include <atomic>

#include "packed_f32x2.cuh"
#include "pet_internal.cuh"

namespace petgb {

static std::atomic<long long> g_launches{0};
void note_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ----------------------------------------------------------------- helpers
__device__ __forceinline__ void kahan_add(float &sum, float &c, float v) {
  const float yk = v - c;
  const float tk = sum + yk;
  c = (tk - sum) - yk;
  sum = tk;
}

__device__ __forceinline__ float bilinear(const float *__restrict__ img, const Samp &S, int plane) {
  const float v00 = (S.z0 && S.b0) ? __ldg(img + S.base) : 0.f;
  const float v01 = (S.z0 && S.b1) ? __ldg(img + S.base + 1) : 0.f;
  const float v10 = (S.z1 && S.b0) ? __ldg(img + S.base + plane) : 0.f;
  const float v11 = (S.z1 && S.b1) ? __ldg(img + S.base + plane + 1) : 0.f;
  return (1.f - S.wz) * ((1.f - S.wb) * v00 + S.wb * v01) + S.wz * ((1.f - S.wb) * v10 + S.wb * v11);
}

__device__ __forceinline__ void scatter(float *__restrict__ g, const Samp &S, int plane, float val) {
  const float a0 = (1.f - S.wz) * val, a1 = S.wz * val;
  if (S.z0 && S.b0) atomicAdd(g + S.base, (1.f - S.wb) * a0);
  if (S.z0 && S.b1) atomicAdd(g + S.base + 1, S.wb * a0);
  if (S.z1 && S.b0) atomicAdd(g + S.base + plane, (1.f - S.wb) * a1);
  if (S.z1 && S.b1) atomicAdd(g + S.base + plane + 1, S.wb * a1);
}

// Number of TOF bins known at compile time (1: non-TOF; 11, 13: exact; 16, 32: bound).
template <int TT>
__device__ __forceinline__ int tof_bins(const DevPlan &P) {
  return (TT == 1 || TT == 11 || TT == 13) ? TT : P.T;
}

// Forward: acc[b] = sum over samples of bilinear(x) * w_b(t) (compensated); the step
// length L is applied by the caller.
template <int TT, int STRIDE = 1>
__device__ __forceinline__ void forward_lor(const DevPlan &P, const Lor &L,
                                            const float *__restrict__ img, float (&acc)[TT],
                                            bool act = true, int off = 0, const float *tab = nullptr) {
  const int Na = L.xdrive ? P.nx : P.ny;
  const int Nb = L.xdrive ? P.ny : P.nx;
  const int plane = Na * Nb;
  const int T = tof_bins<TT>(P);
  float cmp[TT];
#pragma unroll
  for (int b = 0; b < TT; ++b) { acc[b] = 0.f; cmp[b] = 0.f; }
  const float du = P.tof_w * P.tof_inv;
  for (int i = L.i0 + off; i <= L.i1; i += STRIDE) {
    if (!act || i >= Na) continue;
    Samp S;
    sample_at(L, i, Na, Nb, P.nz, S);
    const float val = bilinear(img, S, plane);
    if (TT == 1) {
      kahan_add(acc[0], cmp[0], val);
    } else {
      const float t = fmaf((float)i, L.dt, L.t0);
      const float u0 = (P.tof_e0 - t) * P.tof_inv;
      float uprev = u0, Gprev = tof_edge_G(P, tab, u0);
#pragma unroll
      for (int k = 1; k <= TT; ++k) {
        if (k <= T) {
          const float u = fmaf((float)k, du, u0);
          const float G = tof_edge_G(P, tab, u);
          const float w = tof_bin_weight(P, uprev, Gprev, u, G);
          kahan_add(acc[k - 1], cmp[k - 1], val * w);
          uprev = u;
          Gprev = G;
        }
      }
    }
  }
}

// Back: scatter sum_b q[b] w_b(t) * bilinear weights; q already includes m and L.
template <int TT, int STRIDE = 1>
__device__ __forceinline__ void back_lor(const DevPlan &P, const Lor &L, float *__restrict__ img,
                                         const float (&q)[TT], bool act = true, int off = 0,
                                         const float *tab = nullptr) {
  const int Na = L.xdrive ? P.nx : P.ny;
  const int Nb = L.xdrive ? P.ny : P.nx;
  const int plane = Na * Nb;
  const int T = tof_bins<TT>(P);
  const float du = P.tof_w * P.tof_inv;
  for (int i = L.i0 + off; i <= L.i1; i += STRIDE) {
    if (!act || i >= Na) continue;
    Samp S;
    sample_at(L, i, Na, Nb, P.nz, S);
    float val;
    if (TT == 1) {
      val = q[0];
    } else {
      const float t = fmaf((float)i, L.dt, L.t0);
      const float u0 = (P.tof_e0 - t) * P.tof_inv;
      float uprev = u0, Gprev = tof_edge_G(P, tab, u0);
      val = 0.f;
#pragma unroll
      for (int k = 1; k <= TT; ++k) {
        if (k <= T) {
          const float u = fmaf((float)k, du, u0);
          const float G = tof_edge_G(P, tab, u);
          val = fmaf(q[k - 1], tof_bin_weight(P, uprev, Gprev, u, G), val);
          uprev = u;
          Gprev = G;
        }
      }
    }
    if (val != 0.f) scatter(img, S, plane, val);
  }
}

struct LorIdx {
  int v, p, r, l;
  bool ok;
};

__device__ __forceinline__ LorIdx lor_index(const DevPlan &P, int subset, long long l) {
  LorIdx o;
  const int nsub = subset < 0 ? 1 : P.nsub;
  const int s = subset < 0 ? 0 : subset;
  const int nv = (P.nview - s + nsub - 1) / nsub;
  const long long per_view = (long long)P.nplane * P.nrad;
  o.ok = l < (long long)nv * per_view;
  if (!o.ok) return o;
  o.r = (int)(l % P.nrad);
  const long long t = l / P.nrad;
  o.p = (int)(t % P.nplane);
  const int jv = (int)(t / P.nplane);
  o.v = s + jv * nsub;
  o.l = (int)l;
  return o;
}

// ----------------------------------------------------------------- kernels
template <int TT>
__global__ void __launch_bounds__(kBlock) k_forward(DevPlan P, int subset, const float *__restrict__ x,
                                                    const float *__restrict__ xT, float *__restrict__ out) {
  __shared__ float s_tab[TT > 1 ? kErfcTab + 1 : 1];
  if (TT > 1) load_erfc_tab(P, s_tab);
  const LorIdx id = lor_index(P, subset, (long long)blockIdx.x * blockDim.x + threadIdx.x);
  Lor L = {};
  if (id.ok) lor_setup(P, id.v, id.p, id.r, L);
  warp_uniform_range(L, id.ok);
  float acc[TT];
  forward_lor<TT>(P, L, L.xdrive ? xT : x, acc, id.ok, 0, s_tab);
  if (!id.ok) return;
  const int T = tof_bins<TT>(P);
  const float m = __ldg(&P.m[((size_t)id.v * P.nplane + id.p) * P.nrad + id.r]) * L.L;
#pragma unroll
  for (int b = 0; b < TT; ++b)
    if (b < T) out[(size_t)id.l * T + b] = acc[b] * m;
}

template <int TT>
__global__ void __launch_bounds__(kBlock) k_back(DevPlan P, int subset, const float *__restrict__ q,
                                                 float *__restrict__ g, float *__restrict__ gT) {
  __shared__ float s_tab[TT > 1 ? kErfcTab + 1 : 1];
  if (TT > 1) load_erfc_tab(P, s_tab);
  const LorIdx id = lor_index(P, subset, (long long)blockIdx.x * blockDim.x + threadIdx.x);
  Lor L = {};
  if (id.ok) lor_setup(P, id.v, id.p, id.r, L);
  warp_uniform_range(L, id.ok);
  const int T = tof_bins<TT>(P);
  float qq[TT];
  bool any = false;
  if (id.ok) {
    const float m = __ldg(&P.m[((size_t)id.v * P.nplane + id.p) * P.nrad + id.r]) * L.L;
#pragma unroll
    for (int b = 0; b < TT; ++b) {
      qq[b] = b < T ? __ldg(&q[(size_t)id.l * T + b]) * m : 0.f;
      any |= qq[b] != 0.f;
    }
  }
  back_lor<TT>(P, L, L.xdrive ? gT : g, qq, any, 0, s_tab);
}

__device__ __forceinline__ void block_sum_store(double v, double *out) {
  __shared__ double red[kBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) *out = v;
  }
}

// Fused subset gradient: forward, KL ratio, backprojection; optional FP64 KL partials.
// The block covers kBlock/SPLIT LORs; part j of the block (warps j*W .. (j+1)*W-1)
// takes the planes i = i0 + j, i0 + j + SPLIT, ... of the warp-uniform plane range, so
// the parts carry equal work.  The forward partial sums are exchanged through shared
// memory at a block barrier and added in a fixed order, so every part sees the same
// ybar; each part then backprojects its own planes.  SPLIT multiplies the parallelism of launches with few
// LORs (one subset of a small scanner).
template <int TT, int SPLIT>
__global__ void __launch_bounds__(kBlock) k_grad(DevPlan P, int subset, const int *subset_dev,
                                                 const float *__restrict__ x, const float *__restrict__ xT,
                                                 float *__restrict__ g, float *__restrict__ gT,
                                                 double *__restrict__ kl_part, int mode) {
  constexpr int LPB = kBlock / SPLIT;  // LORs per block
  __shared__ float xs[SPLIT > 1 ? SPLIT : 1][SPLIT > 1 ? LPB : 1][TT];
  __shared__ float s_tab[TT > 1 ? kErfcTab + 1 : 1];
  if (TT > 1) load_erfc_tab(P, s_tab);
  if (subset_dev) subset = *subset_dev;
  const int part = threadIdx.x / LPB;
  const int tl = threadIdx.x % LPB;
  const LorIdx id = lor_index(P, subset, (long long)blockIdx.x * LPB + tl);
  double kl = 0.0;
  Lor L = {};
  if (id.ok) lor_setup(P, id.v, id.p, id.r, L);
  warp_uniform_range(L, id.ok);
  float acc[TT];
  if (mode != MODE_SENS) {
    forward_lor<TT, SPLIT>(P, L, L.xdrive ? xT : x, acc, id.ok, part, s_tab);
    if (SPLIT > 1) {
#pragma unroll
      for (int b = 0; b < TT; ++b) xs[part][tl][b] = acc[b];
      __syncthreads();
#pragma unroll
      for (int b = 0; b < TT; ++b) {
        float t = xs[0][tl][b];
#pragma unroll
        for (int j = 1; j < SPLIT; ++j) t += xs[j][tl][b];
        acc[b] = t;
      }
    }
  }
  float q[TT];
  bool any = false;
  {
    const int T = tof_bins<TT>(P);
    const size_t lor = id.ok ? ((size_t)id.v * P.nplane + id.p) * P.nrad + id.r : 0;
    const float mL = id.ok ? __ldg(&P.m[lor]) * L.L : 0.f;
#pragma unroll
    for (int b = 0; b < TT; ++b) {
      q[b] = 0.f;
      if (b < T && id.ok) {
        if (mode == MODE_SENS) {
          q[b] = mL;
        } else {
          const size_t bi = lor * T + b;
          const float ybar = fmaf(mL, acc[b], __ldg(&P.r[bi]));
          const float yb = load_y(P, bi);
          const bool count = kl_part && part == 0;
          if (!(ybar > 0.f)) {
            if (yb > 0.f) atomicOr(P.err, 1);
            q[b] = (grad_like(mode) && yb == 0.f) ? mL : 0.f;
            if (count && yb == 0.f) kl += (double)fmaxf(ybar, 0.f);
          } else {
            if (grad_like(mode)) q[b] = mL * (1.f - yb / ybar);
            else if (mode == MODE_EM) q[b] = mL * (yb / ybar);
            if (count) {
              const double db = ybar, dy = yb;
              kl += (yb > 0.f) ? (db - dy + dy * log(dy / db)) : db;
            }
          }
        }
        if (mode == MODE_NGRAD) q[b] = -q[b];
        any |= q[b] != 0.f;
      }
    }
  }
  if (mode != MODE_OBJ) back_lor<TT, SPLIT>(P, L, L.xdrive ? gT : g, q, any, part, s_tab);
  if (kl_part) block_sum_store(kl, kl_part + blockIdx.x);
}

// Multi-plane fused subset gradient (non-TOF): each thread owns K consecutive planes of
// one (view, radial bin).  The in-plane sample position (fb, its floor and weight) is
// shared by the K LORs, each plane adds only its axial coordinate; the K accumulation
// chains are independent, which keeps more loads in flight per thread.  Parts (SPLIT)
// interleave the planes i exactly as in k_grad.  Per LOR the arithmetic is that of
// k_grad<1, SPLIT>.
template <int K, int SPLIT>
__device__ __forceinline__ void grad_mp_body(const DevPlan &P, int subset, int blk,
                                             const float *__restrict__ x, const float *__restrict__ xT,
                                             float *__restrict__ g, float *__restrict__ gT,
                                             double *__restrict__ kl_out, int mode) {
  constexpr int LPB = kBlock / SPLIT;
  __shared__ float xs[SPLIT > 1 ? SPLIT : 1][SPLIT > 1 ? LPB : 1][K];
  const int part = threadIdx.x / LPB;
  const int tl = threadIdx.x % LPB;
  const int nsub = subset < 0 ? 1 : P.nsub;
  const int s0 = subset < 0 ? 0 : subset;
  const int nv = (P.nview - s0 + nsub - 1) / nsub;
  const int npg = (P.nplane + K - 1) / K;
  const long long u = (long long)blk * LPB + tl;
  const bool ok = u < (long long)nv * npg * P.nrad;
  int v = 0, r = 0, p0 = 0;
  if (ok) {
    r = (int)(u % P.nrad);
    const long long t = u / P.nrad;
    p0 = (int)(t % npg) * K;
    v = s0 + (int)(t / npg) * nsub;
  }
  // shared in-plane geometry (lor_setup for the K planes at once)
  const float4 vw = __ldg(&P.view[v]);
  const float4 vr = __ldg(&P.vr[v * P.nrad + r]);
  const bool xdrive = vw.x != 0.f;
  const float dfb = vw.y, dau = vw.z, fb0 = vr.x, t0b = vr.y, inv2h = vr.z;
  const float g1 = dau * inv2h, g2 = t0b * inv2h;
  const int Na = xdrive ? P.nx : P.ny;
  const int Nb = xdrive ? P.ny : P.nx;
  const int plane = Na * Nb;
  float fz0[K], dfz[K], Lk[K];
  bool pv[K];
  float lo_b = 0.f, hi_b = (float)(Na - 1);
  clip_range(fb0, dfb, -1.f, (float)Nb, lo_b, hi_b);
  float lo = 1e30f, hi = -1e30f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int p = p0 + k;
    pv[k] = ok && p < P.nplane;
    const float4 pl = __ldg(&P.plane[pv[k] ? p : 0]);
    dfz[k] = g1 * pl.y;
    fz0[k] = fmaf(g2, pl.y, pl.x);
    const float kk = pl.z * inv2h;
    Lk[k] = fabsf(dau) * sqrtf(fmaf(kk, kk, 1.f));
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
  const float *img = xdrive ? xT : x;
  float acc[K], cmp[K];
#pragma unroll
  for (int k = 0; k < K; ++k) { acc[k] = 0.f; cmp[k] = 0.f; }
  if (mode != MODE_SENS) {
    for (int i = L.i0 + part; i <= L.i1; i += SPLIT) {
      if (!ok || i >= Na) continue;
      const float fb = fmaf((float)i, dfb, fb0);
      const float fbf = floorf(fb);
      const int ib = (int)fbf;
      const float wb = fb - fbf;
      const bool b0 = (unsigned)ib < (unsigned)Nb;
      const bool b1 = (unsigned)(ib + 1) < (unsigned)Nb && wb != 0.f;
      const int row = i * Nb + ib;
      // bilinear interpolation: the two rows of each plane as one packed pair, then the
      // axial step for two planes at a time
      const float2 wbb = make_float2(wb, wb), wbb1 = make_float2(1.f - wb, 1.f - wb);
      float2 h[K];
      float wzk[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float fz = fmaf((float)i, dfz[k], fz0[k]);
        const float fzf = floorf(fz);
        const int iz = (int)fzf;
        const float wz = fz - fzf;
        const bool z0 = pv[k] && (unsigned)iz < (unsigned)P.nz;
        const bool z1 = pv[k] && (unsigned)(iz + 1) < (unsigned)P.nz && wz != 0.f;
        const int base = iz * plane + row;
        const float v00 = (z0 && b0) ? __ldg(img + base) : 0.f;
        const float v01 = (z0 && b1) ? __ldg(img + base + 1) : 0.f;
        const float v10 = (z1 && b0) ? __ldg(img + base + plane) : 0.f;
        const float v11 = (z1 && b1) ? __ldg(img + base + plane + 1) : 0.f;
        h[k] = fma2(wbb, make_float2(v01, v11), mul2(wbb1, make_float2(v00, v10)));
        wzk[k] = wz;
      }
      if (K == 1) {
        kahan_add(acc[0], cmp[0], fmaf(wzk[0], h[0].y, (1.f - wzk[0]) * h[0].x));
      } else {
#pragma unroll
        for (int k = 0; k + 1 < K; k += 2) {
          const float2 wz2 = make_float2(wzk[k], wzk[k + 1]);
          const float2 r2 = fma2(wz2, make_float2(h[k].y, h[k + 1].y),
                                 mul2(sub2(make_float2(1.f, 1.f), wz2), make_float2(h[k].x, h[k + 1].x)));
          kahan_add(acc[k], cmp[k], r2.x);
          kahan_add(acc[k + 1], cmp[k + 1], r2.y);
        }
      }
    }
    if (SPLIT > 1) {
#pragma unroll
      for (int k = 0; k < K; ++k) xs[part][tl][k] = acc[k];
      __syncthreads();
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float t = xs[0][tl][k];
#pragma unroll
        for (int j = 1; j < SPLIT; ++j) t += xs[j][tl][k];
        acc[k] = t;
      }
    }
  }
  double kl = 0.0;
  float q[K];
  bool any = false;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    q[k] = 0.f;
    if (!pv[k]) continue;
    const size_t lor = ((size_t)v * P.nplane + p0 + k) * P.nrad + r;
    const float mL = __ldg(&P.m[lor]) * Lk[k];
    if (mode == MODE_SENS) {
      q[k] = mL;
    } else {
      const float ybar = fmaf(mL, acc[k], __ldg(&P.r[lor]));
      const float yb = load_y(P, lor);
      const bool count = kl_out && part == 0;
      if (!(ybar > 0.f)) {
        if (yb > 0.f) atomicOr(P.err, 1);
        q[k] = (grad_like(mode) && yb == 0.f) ? mL : 0.f;
        if (count && yb == 0.f) kl += (double)fmaxf(ybar, 0.f);
      } else {
        if (grad_like(mode)) q[k] = mL * (1.f - yb / ybar);
        else if (mode == MODE_EM) q[k] = mL * (yb / ybar);
        if (count) {
          const double db = ybar, dy = yb;
          kl += (yb > 0.f) ? (db - dy + dy * log(dy / db)) : db;
        }
      }
    }
    if (mode == MODE_NGRAD) q[k] = -q[k];
    any |= q[k] != 0.f;
  }
  if (mode != MODE_OBJ) {
    float *out = xdrive ? gT : g;
    for (int i = L.i0 + part; i <= L.i1; i += SPLIT) {
      if (!any || i >= Na) continue;
      const float fb = fmaf((float)i, dfb, fb0);
      const float fbf = floorf(fb);
      const int ib = (int)fbf;
      const float wb = fb - fbf;
      const bool b0 = (unsigned)ib < (unsigned)Nb;
      const bool b1 = (unsigned)(ib + 1) < (unsigned)Nb && wb != 0.f;
      const int row = i * Nb + ib;
      const float2 wbp = make_float2(1.f - wb, wb);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (q[k] == 0.f) continue;
        const float fz = fmaf((float)i, dfz[k], fz0[k]);
        const float fzf = floorf(fz);
        const int iz = (int)fzf;
        const float wz = fz - fzf;
        const bool z0 = (unsigned)iz < (unsigned)P.nz;
        const bool z1 = (unsigned)(iz + 1) < (unsigned)P.nz && wz != 0.f;
        const int base = iz * plane + row;
        const float2 a = mul2(make_float2(1.f - wz, wz), make_float2(q[k], q[k]));
        const float2 lo2 = mul2(wbp, make_float2(a.x, a.x));
        const float2 up2 = mul2(wbp, make_float2(a.y, a.y));
        if (z0 && b0) atomicAdd(out + base, lo2.x);
        if (z0 && b1) atomicAdd(out + base + 1, lo2.y);
        if (z1 && b0) atomicAdd(out + base + plane, up2.x);
        if (z1 && b1) atomicAdd(out + base + plane + 1, up2.y);
      }
    }
  }
  if (kl_out) block_sum_store(kl, kl_out);
}

template <int K, int SPLIT>
__global__ void __launch_bounds__(kBlock) k_grad_mp(DevPlan P, int subset, const int *subset_dev,
                                                    const float *__restrict__ x, const float *__restrict__ xT,
                                                    float *__restrict__ g, float *__restrict__ gT,
                                                    double *__restrict__ kl_part, int mode) {
  if (subset_dev) subset = *subset_dev;
  grad_mp_body<K, SPLIT>(P, subset, blockIdx.x, x, xT, g, gT, kl_part ? kl_part + blockIdx.x : nullptr, mode);
}

// Index of the job owning this block: jobs own consecutive block ranges starting at
// begin[j] (begin[njobs] = total blocks).  One warp compares 32 offsets per step.
__device__ __forceinline__ int find_job(const int *__restrict__ begin, int njobs) {
  __shared__ int s_job;
  if (threadIdx.x < 32) {
    int job = 0;
    for (int base = 0; base < njobs; base += 32) {
      const int j = base + (int)threadIdx.x;
      const bool le = j < njobs && __ldg(&begin[j]) <= (int)blockIdx.x;
      const unsigned m = __ballot_sync(0xffffffffu, le);
      job = base + __popc(m) - 1;
      if (m != 0xffffffffu) break;
    }
    if (threadIdx.x == 0) s_job = job;
  }
  __syncthreads();
  return s_job;
}

// Batched fused gradient: one launch covers the current subset of every job.
template <int K, int SPLIT>
__global__ void __launch_bounds__(kBlock) k_grad_mp_batch(const GradJob *__restrict__ jobs,
                                                          const int *__restrict__ begin, int njobs, int mode) {
  __shared__ GradJob sj;
  const int j = find_job(begin, njobs);
  if (threadIdx.x == 0) sj = jobs[j];
  __syncthreads();
  const int subset = *sj.subset_dev;
  if (subset == kBatchSkip) return;  // this instance runs the window alone (whole block)
  grad_mp_body<K, SPLIT>(sj.P, subset, (int)blockIdx.x - __ldg(&begin[j]), sj.x, sj.xT, sj.g, sj.gT, nullptr, mode);
}

cudaError_t launch_grad_batch(const GradJob *jobs, const int *begin, int njobs, int total_blocks, int K,
                              int split, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  note_launch();
#define PET_GB(KK, SP) k_grad_mp_batch<KK, SP><<<total_blocks, kBlock, 0, st>>>(jobs, begin, njobs, MODE_GRAD)
  if (K == 4) {
    if (split == 8) PET_GB(4, 8); else if (split == 4) PET_GB(4, 4); else if (split == 2) PET_GB(4, 2); else PET_GB(4, 1);
  } else if (K == 2) {
    if (split == 8) PET_GB(2, 8); else if (split == 4) PET_GB(2, 4); else if (split == 2) PET_GB(2, 2); else PET_GB(2, 1);
  } else {
    if (split == 8) PET_GB(1, 8); else if (split == 4) PET_GB(1, 4); else if (split == 2) PET_GB(1, 2); else PET_GB(1, 1);
  }
#undef PET_GB
  return cudaGetLastError();
}

int grad_blocks_shape(const DevPlan &P, int nv, int K, int split) {
  const long long units = (long long)nv * ((P.nplane + K - 1) / K) * P.nrad;
  const int lpb = kBlock / split;
  return (int)((units + lpb - 1) / lpb);
}

// m = sens * exp(-P mu) for every LOR (non-TOF forward of the attenuation image).
__global__ void __launch_bounds__(kBlock) k_mult(DevPlan P, const float *__restrict__ mu,
                                                 const float *__restrict__ muT,
                                                 const float *__restrict__ sens, float *__restrict__ m) {
  const LorIdx id = lor_index(P, -1, (long long)blockIdx.x * blockDim.x + threadIdx.x);
  float s = (sens && id.ok) ? __ldg(&sens[id.l]) : 1.f;
  if (mu) {
    Lor L = {};
    if (id.ok) lor_setup(P, id.v, id.p, id.r, L);
    warp_uniform_range(L, id.ok);
    float acc[1];
    forward_lor<1>(P, L, L.xdrive ? muT : mu, acc, id.ok);
    s *= expf(-acc[0] * L.L);
  }
  if (id.ok) m[id.l] = s;
}

// Tiled transpose of each z-slice: src [z][A][B] -> dst [z][B][A].  accumulate: 0 writes,
// 1 adds, 2 adds and clears the source tile (keeps an accumulator zeroed between uses).
__global__ void k_transpose(float *__restrict__ src, float *__restrict__ dst, int A, int B,
                            int accumulate) {
  __shared__ float tile[32][33];
  const int z = blockIdx.z;
  const int b0 = blockIdx.x * 32, a0 = blockIdx.y * 32;
  const size_t off = (size_t)z * A * B;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int a = a0 + j, b = b0 + threadIdx.x;
    if (a < A && b < B) {
      tile[j][threadIdx.x] = src[off + (size_t)a * B + b];
      if (accumulate == 2) src[off + (size_t)a * B + b] = 0.f;
    }
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int b = b0 + j, a = a0 + threadIdx.x;
    if (a < A && b < B) {
      const size_t o = off + (size_t)b * A + a;
      dst[o] = accumulate ? dst[o] + tile[threadIdx.x][j] : tile[threadIdx.x][j];
    }
  }
}

// Voxel-driven deterministic backprojection: each thread gathers, in a fixed order
// with compensated summation, every (LOR, sample) whose bilinear footprint covers its
// voxel.  The sample positions are computed with exactly the arithmetic of
// lor_setup/sample_at, so the weights are those of the ray-driven pair.  ones != 0
// backprojects q = 1 (sensitivity A^T 1).
template <int TT>
__global__ void __launch_bounds__(kBlock) k_back_det(DevPlan P, DevPlanDet D, int subset,
                                                     const float *__restrict__ q, float *__restrict__ g,
                                                     int ones) {
  __shared__ float s_tab[TT > 1 ? kErfcTab + 1 : 1];
  if (TT > 1) load_erfc_tab(P, s_tab);
  const float *tab = s_tab;
  const int nvox = P.nx * P.ny * P.nz;
  const int vox = blockIdx.x * blockDim.x + threadIdx.x;
  if (vox >= nvox) return;
  const int ix = vox % P.nx, iy = (vox / P.nx) % P.ny, iz = vox / (P.nx * P.ny);
  const int nsub = subset < 0 ? 1 : P.nsub;
  const int s0 = subset < 0 ? 0 : subset;
  const int T = tof_bins<TT>(P);
  const float du = P.tof_w * P.tof_inv;
  float sum = 0.f, cmp = 0.f;
  int jv = 0;
  for (int v = s0; v < P.nview; v += nsub, ++jv) {
    const float4 vw = __ldg(&P.view[v]);
    const bool xd = vw.x != 0.f;
    const int i = xd ? ix : iy, j = xd ? iy : ix;
    const float dfb = vw.y, dau = vw.z;
    const float2 aff = __ldg(&D.view_aff[v]);
    const float base = fmaf((float)i, dfb, aff.x);
    const float ra = ((float)(j - 1) - base) / aff.y, rb = ((float)(j + 1) - base) / aff.y;
    const int r0 = max(0, (int)floorf(fmaxf(fminf(ra, rb), -4.f)) - 1);
    const int r1 = min(P.nrad - 1, (int)ceilf(fminf(fmaxf(ra, rb), (float)P.nrad + 4.f)) + 1);
    for (int r = r0; r <= r1; ++r) {
      const float4 vr = __ldg(&P.vr[v * P.nrad + r]);
      const float fb = fmaf((float)i, dfb, vr.x);
      const float fbf = floorf(fb);
      const int ib = (int)fbf;
      const float wb = fb - fbf;
      float wbj;
      if (ib == j) wbj = 1.f - wb;
      else if (ib + 1 == j) wbj = wb;
      else continue;
      const float t0b = vr.y, inv2h = vr.z;
      const float g1 = dau * inv2h, g2 = t0b * inv2h;
      const float cz = fmaf((float)i, g1, g2);  // fz ~ zs + zd * cz
      for (int gi = 0; gi < D.ngroups; ++gi) {
        const int2 gr = __ldg(&D.groups[gi]);
        const float zd = __ldg(&D.gzd[gi]);
        const float lo_zs = (float)(iz - 1) - zd * cz - 1e-3f;
        const float hi_zs = (float)(iz + 1) - zd * cz + 1e-3f;
        int a = gr.x, b = gr.x + gr.y;  // first zs >= lo_zs
        while (a < b) {
          const int mid = (a + b) >> 1;
          if (__ldg(&D.gzs[mid]) < lo_zs) a = mid + 1;
          else b = mid;
        }
        for (int kq = a; kq < gr.x + gr.y && __ldg(&D.gzs[kq]) <= hi_zs; ++kq) {
        const int p = __ldg(&D.gplane[kq]);
        const float4 pl = __ldg(&P.plane[p]);
        const float dfz = g1 * pl.y;
        const float fz0 = fmaf(g2, pl.y, pl.x);
        const float fz = fmaf((float)i, dfz, fz0);
        const float fzf = floorf(fz);
        const int jz = (int)fzf;
        const float wz = fz - fzf;
        float wzk;
        if (jz == iz) wzk = 1.f - wz;
        else if (jz + 1 == iz) wzk = wz;
        else continue;
        const float kk = pl.z * inv2h;
        const float sec = sqrtf(fmaf(kk, kk, 1.f));
        const float mL = __ldg(&P.m[((size_t)v * P.nplane + p) * P.nrad + r]) * (fabsf(dau) * sec);
        const size_t ql = (((size_t)jv * P.nplane + p) * P.nrad + r) * T;
        float val;
        if (TT == 1) {
          val = ones ? 1.f : __ldg(&q[ql]);
        } else {
          const float t = fmaf((float)i, dau * sec, t0b * sec);
          const float u0 = (P.tof_e0 - t) * P.tof_inv;
          float uprev = u0, Gprev = tof_edge_G(P, tab, u0);
          val = 0.f;
#pragma unroll
          for (int k = 1; k <= TT; ++k) {
            if (k <= T) {
              const float u = fmaf((float)k, du, u0);
              const float G = tof_edge_G(P, tab, u);
              const float qb = ones ? 1.f : __ldg(&q[ql + k - 1]);
              val = fmaf(qb, tof_bin_weight(P, uprev, Gprev, u, G), val);
              uprev = u;
              Gprev = G;
            }
          }
        }
        kahan_add(sum, cmp, mL * val * (wbj * wzk));
        }
      }
    }
  }
  g[vox] = sum;
}

// KL ratio on a compact subset sinogram holding A_s x: mode MODE_GRAD writes
// 1 - y/ybar, MODE_EM y/ybar; optional FP64 KL partial sums per block.
__global__ void __launch_bounds__(kBlock) k_ratio(DevPlan P, int subset, const float *__restrict__ ax,
                                                  float *__restrict__ q, double *__restrict__ kl_part,
                                                  int mode) {
  const int T = P.T > 1 ? P.T : 1;
  const long long bin = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const LorIdx id = lor_index(P, subset, bin / T);
  double kl = 0.0;
  if (id.ok) {
    const int b = (int)(bin % T);
    const size_t bi = (((size_t)id.v * P.nplane + id.p) * P.nrad + id.r) * T + b;
    const float ybar = ax[bin] + __ldg(&P.r[bi]);
    const float yb = load_y(P, bi);
    float qq;
    if (!(ybar > 0.f)) {
      if (yb > 0.f) atomicOr(P.err, 1);
      qq = (mode == MODE_GRAD && yb == 0.f) ? 1.f : 0.f;
      if (yb == 0.f) kl = (double)fmaxf(ybar, 0.f);
    } else {
      qq = mode == MODE_GRAD ? 1.f - yb / ybar : yb / ybar;
      const double db = ybar, dy = yb;
      kl = (yb > 0.f) ? (db - dy + dy * log(dy / db)) : db;
    }
    if (q) q[bin] = qq;
  }
  if (kl_part) block_sum_store(kl, kl_part + blockIdx.x);
}

__global__ void k_fill(float *__restrict__ p, size_t n, float v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// ----------------------------------------------------------------- launchers
// TOF plans with a register window use the windowed kernel (tof_kernels.cu: 1 or 2 planes
// per thread, up to 8 parts); other TOF plans the kernels with per-edge weights.
static bool use_tofk(const DevPlan &P) { return P.T > 1 && tofk_supported(P, 1); }

cudaError_t launch_fill(float *p, size_t n, float v, cudaStream_t st) {
  note_launch();
  k_fill<<<(unsigned)std::min<size_t>(2432, (n + 255) / 256), 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

static int views_in(const DevPlan &P, int subset) {
  if (subset < 0) return P.nview;
  return (P.nview - subset + P.nsub - 1) / P.nsub;
}

static unsigned blocks_for(const DevPlan &P, int nviews) {
  const long long n = (long long)nviews * P.nplane * P.nrad;
  return (unsigned)((n + kBlock - 1) / kBlock);
}


#define PET_TOF_DISPATCH(KERNEL, GRID, STREAM, ...)                             \
  do {                                                                         \
    note_launch();                                                             \
    if (P.T <= 1) KERNEL<1><<<GRID, kBlock, 0, STREAM>>>(__VA_ARGS__);         \
    else if (P.T == 11) KERNEL<11><<<GRID, kBlock, 0, STREAM>>>(__VA_ARGS__);  \
    else if (P.T == 13) KERNEL<13><<<GRID, kBlock, 0, STREAM>>>(__VA_ARGS__);  \
    else if (P.T <= 16) KERNEL<16><<<GRID, kBlock, 0, STREAM>>>(__VA_ARGS__);  \
    else KERNEL<32><<<GRID, kBlock, 0, STREAM>>>(__VA_ARGS__);                 \
  } while (0)

cudaError_t launch_forward(const DevPlan &P, int subset, const float *x, const float *xT,
                           float *out, cudaStream_t st) {
  const unsigned grid = blocks_for(P, views_in(P, subset));
  if (grid == 0) return cudaSuccess;
  PET_TOF_DISPATCH(k_forward, grid, st, P, subset, x, xT, out);
  return cudaGetLastError();
}

cudaError_t launch_back(const DevPlan &P, int subset, const float *q, float *g, float *gT,
                        cudaStream_t st) {
  const unsigned grid = blocks_for(P, views_in(P, subset));
  if (grid == 0) return cudaSuccess;
  PET_TOF_DISPATCH(k_back, grid, st, P, subset, q, g, gT);
  return cudaGetLastError();
}

// Parts per LOR: enough threads for about two full waves (152 SMs x 2048 threads).
static int split_for(long long nlor) {
  const long long target = 2LL * 152 * 2048;
  if (nlor * 2 > target) return 1;
  if (nlor * 4 > target) return 2;
  return 4;
}

int grad_blocks_for(const DevPlan &P, int nv);
int grad_blocks(const DevPlan &P, int max_views) { return grad_blocks_for(P, max_views); }

#define PET_GRAD_LAUNCH(SPLIT)                                                                  \
  do {                                                                                         \
    if (P.T <= 1) k_grad<1, SPLIT><<<grid, kBlock, 0, st>>>(P, subset, subset_dev, x, xT, g, gT, kl_part, mode);   \
    else if (P.T <= 16) k_grad<16, SPLIT><<<grid, kBlock, 0, st>>>(P, subset, subset_dev, x, xT, g, gT, kl_part, mode); \
    else k_grad<32, SPLIT><<<grid, kBlock, 0, st>>>(P, subset, subset_dev, x, xT, g, gT, kl_part, mode);           \
  } while (0)

static int views_for_launch(const DevPlan &P, int subset, const int *subset_dev) {
  return subset_dev ? (P.nview + P.nsub - 1) / P.nsub : views_in(P, subset);
}

// Launch shape of the fused gradient: planes per thread and parts per LOR.  P.grad_k /
// P.grad_split hold the autotuner's choice (0: heuristic).  Largest parts per LOR of a
// launch: 16 without TOF, 8 with the windowed TOF kernel, 4 otherwise.
int max_split(const DevPlan &P) {
  if (P.T <= 1) return 16;
  return use_tofk(P) ? 8 : 4;
}

// Largest planes per thread of the fused gradient: 4 without TOF, 2 with the windowed
// TOF kernel, else 1.
int max_planes(const DevPlan &P) {
  if (P.T <= 1) return 4;
  return tofk_supported(P, 4) ? 4 : (tofk_supported(P, 2) ? 2 : 1);
}

static void grad_shape(const DevPlan &P, long long nlor, int &K, int &split) {
  if (use_tofk(P)) {
    K = P.grad_k > 0 ? P.grad_k : 2;
    if (!tofk_supported(P, K)) K = 1;
    split = P.grad_split > 0 ? P.grad_split : 1;
    split = std::min(split, 8);
    return;
  }
  K = (P.T <= 1 && P.grad_k > 0) ? P.grad_k : 1;
  split = P.grad_split > 0 ? P.grad_split : split_for(nlor);
  split = std::min(split, max_split(P));
}

int grad_blocks_for(const DevPlan &P, int nv) {
  const long long nlor = (long long)nv * P.nplane * P.nrad;
  int K, split;
  grad_shape(P, nlor, K, split);
  if (use_tofk(P)) return tofk_blocks(P, nv, K, split);
  const long long units = (long long)nv * ((P.nplane + K - 1) / K) * P.nrad;
  const int lpb = kBlock / split;
  return (int)((units + lpb - 1) / lpb);
}

#define PET_GRAD_MP(KK, SP) k_grad_mp<KK, SP><<<grid, kBlock, 0, st>>>(P, subset, subset_dev, x, xT, g, gT, kl_part, mode)

cudaError_t launch_grad(const DevPlan &P, int subset, const int *subset_dev, const float *x,
                        const float *xT, float *g, float *gT, double *kl_part, int mode,
                        int *nblocks_out, cudaStream_t st) {
  // with a device-side subset index the grid covers the largest subset
  const int nv = views_for_launch(P, subset, subset_dev);
  const long long nlor = (long long)nv * P.nplane * P.nrad;
  int K, split;
  grad_shape(P, nlor, K, split);
  const unsigned grid = (unsigned)grad_blocks_for(P, nv);
  if (nblocks_out) *nblocks_out = (int)grid;
  if (grid == 0) return cudaSuccess;
  if (use_tofk(P)) return launch_grad_tofk(P, K, split, grid, subset, subset_dev, x, xT, g, gT, kl_part, mode, st);
  note_launch();
  if (K == 4) {
    if (split == 16) PET_GRAD_MP(4, 16);
    else if (split == 8) PET_GRAD_MP(4, 8);
    else if (split == 4) PET_GRAD_MP(4, 4);
    else if (split == 2) PET_GRAD_MP(4, 2);
    else PET_GRAD_MP(4, 1);
  } else if (K == 2) {
    if (split == 16) PET_GRAD_MP(2, 16);
    else if (split == 8) PET_GRAD_MP(2, 8);
    else if (split == 4) PET_GRAD_MP(2, 4);
    else if (split == 2) PET_GRAD_MP(2, 2);
    else PET_GRAD_MP(2, 1);
  } else if (split == 16) {
    k_grad<1, 16><<<grid, kBlock, 0, st>>>(P, subset, subset_dev, x, xT, g, gT, kl_part, mode);
  } else if (split == 8) {
    k_grad<1, 8><<<grid, kBlock, 0, st>>>(P, subset, subset_dev, x, xT, g, gT, kl_part, mode);
  } else if (split == 4) {
    PET_GRAD_LAUNCH(4);
  } else if (split == 2) {
    PET_GRAD_LAUNCH(2);
  } else {
    PET_GRAD_LAUNCH(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_back_det(const DevPlan &P, const DevPlanDet &D, int subset, const float *q,
                            float *g, int ones, cudaStream_t st) {
  const long long nvox = (long long)P.nx * P.ny * P.nz;
  const unsigned grid = (unsigned)((nvox + kBlock - 1) / kBlock);
  PET_TOF_DISPATCH(k_back_det, grid, st, P, D, subset, q, g, ones);
  return cudaGetLastError();
}

int ratio_blocks(const DevPlan &P, int subset) {
  const long long n = (long long)views_in(P, subset) * P.nplane * P.nrad * (P.T > 1 ? P.T : 1);
  return (int)((n + kBlock - 1) / kBlock);
}

cudaError_t launch_ratio(const DevPlan &P, int subset, const float *ax, float *q, double *kl_part,
                         int mode, cudaStream_t st) {
  const int grid = ratio_blocks(P, subset);
  if (grid == 0) return cudaSuccess;
  note_launch();
  k_ratio<<<grid, kBlock, 0, st>>>(P, subset, ax, q, kl_part, mode);
  return cudaGetLastError();
}

cudaError_t launch_mult(const DevPlan &P, const float *mu, const float *muT, const float *sens,
                        float *m, cudaStream_t st) {
  const unsigned grid = blocks_for(P, P.nview);
  note_launch();
  k_mult<<<grid, kBlock, 0, st>>>(P, mu, muT, sens, m);
  return cudaGetLastError();
}

cudaError_t launch_transpose(const float *src, float *dst, int nx, int ny, int nz, int to_xfast,
                             int accumulate, cudaStream_t st) {
  // to_xfast = 0: x[z][y][x] -> xT[z][x][y]  (A = ny, B = nx)
  // to_xfast = 1: xT[z][x][y] -> x[z][y][x]  (A = nx, B = ny)
  const int A = to_xfast ? nx : ny, B = to_xfast ? ny : nx;
  dim3 grid((B + 31) / 32, (A + 31) / 32, nz), block(32, 8);
  note_launch();
  k_transpose<<<grid, block, 0, st>>>(const_cast<float *>(src), dst, A, B, accumulate);
  return cudaGetLastError();
}

}  // namespace petgb
