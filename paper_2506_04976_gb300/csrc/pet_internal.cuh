// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pet_gb300.h"

namespace petgb {

constexpr int kBlock = 256;
// Entries of the erfc table used for TOF bin edges: linear interpolation of erfc on
// [0, 3/sqrt 2] with step h = amax/4096 has error <= h^2/8 max|erfc''| < 3.3e-8.
constexpr int kErfcTab = 4096;

// Device view of a plan, passed to kernels by value.
//
// LOR geometry is stored in the "driving frame" of its view: a is the in-plane axis
// along which Joseph's method steps (one sample per voxel-centre plane a_i), b the
// other in-plane axis.  Views driven along x read/write the image through a
// transposed copy [z][x][y] so that adjacent radial bins (adjacent threads) touch
// adjacent addresses.  Per LOR (v, p, r) the sample at plane i has fractional indices
//   fb(i) = fb0 + i dfb,   fz(i) = (zs + g2 zd) + i (g1 zd),
// with g1 = dau/(2h), g2 = t0b/(2h), position along the LOR from its midpoint
//   t(i) = (t0b + i dau) sec,  sec = sqrt(1 + (dzmm/(2h))^2),
// and step length L = |dau| sec, where dau = delta_a / u_a, t0b = (a_0 - M_a)/u_a,
// M the LOR's closest point to the axis and h its in-plane half-length.
struct DevPlan {
  int nx, ny, nz;
  int nrad, nview, nplane, T;
  int nsub;
  const float4 *view;   // [V]  {xdrive, dfb, dau, 0}
  const float4 *vr;     // [V*R] {fb0, t0b, inv2h, 0}
  const float4 *plane;  // [P]  {zs, zd, dzmm, 0}
  const void *y;
  int yt;
  const float *r;
  const float *m;
  float tof_inv;        // 1 / (sqrt(2) sigma)
  float tof_e0;         // position of bin edge 0 (mm): -T w / 2
  float tof_w;          // bin width (mm)
  float tof_amax;       // truncation 3/sqrt(2) in units of sqrt(2) sigma
  float tof_erfc_amax;  // erfc(amax)
  float tof_half_norm;  // 1 / (2 erf(amax))
  int *err;             // device error word (bit 0: infeasible ybar)
  const float *erfc_tab; // erfc(j amax / kErfcTab), j = 0..kErfcTab (TOF)
  float erfc_scale;      // kErfcTab / amax
  int grad_k;           // fused gradient: planes per thread (0 = heuristic)
  int grad_split;       // fused gradient: parts per LOR (0 = heuristic)
  // windowed TOF kernel (tof_kernels.cu): rows of the interpolated bin-weight table,
  // x' = t' / h + tofw_off is the window coordinate of a sample at (mirrored) position t'
  const float4 *tofw_tab;  // [kTofM][WIN/2] (F_2p, F_2p+1, slope_2p, slope_2p+1), WIN = 4, 6 or 8
  float tofw_inv_h;        // 1 / h, h = bin width / kTofM
  float tofw_off;          // (R - c_0)/h - Ktab + kTofM
  int tofw_win;            // bins a sample can meet (0: no table)
  const int *tof_grp2;     // [tof_ngrp2][2] plane pairs of equal axial slope (-1: none)
  int tof_ngrp2;
  const int *tof_grp4;     // [tof_ngrp4][4] plane quadruples of equal axial slope (-1: none)
  int tof_ngrp4;
  int tof_zint;             // 1: the planes of every group lie a whole number of slices apart
  unsigned long long *tof_work;  // work counter of the persistent TOF kernel (plan scratch)
  int nsm;                       // multiprocessors of the plan's device
  float *tof_xp, *tof_xtp;       // zero-padded image copies in the two view frames (plan scratch)
  float *tof_gp, *tof_gtp;       // zero-padded gradient accumulators in the two view frames
};

// Windowed TOF kernel constants: threads per block, table rows per bin width (a power of
// two), largest number of TOF bins.
constexpr int kTofBlock = 512;
constexpr int kTofLogM = 10;
constexpr int kTofM = 1 << kTofLogM;
constexpr int kTofMaxBins = 16;
constexpr int kTofPad = 2;  // zero voxels on each side of the b and z axes of the padded frames

// Per-view data for the voxel-driven (deterministic) backprojector: fb0 is affine in
// the radial index, fb0(v, r) ~ fbA + r fbB, used only to find candidate LORs.
// Planes are grouped by their axial slope zd (equal FP32 values); within a group they
// are listed by increasing zs, so the planes whose ray can reach a given slice are a
// contiguous run found by binary search.
struct DevPlanDet {
  const float2 *view_aff;  // [V] {fbA, fbB}
  int ngroups;
  const int2 *groups;      // [ngroups] {first index into gplane, count}
  const float *gzd;        // [ngroups] zd of the group
  const int *gplane;       // [P] plane indices, grouped, sorted by zs within a group
  const float *gzs;        // [P] zs of gplane[k]
};

struct Lor {
  int xdrive;
  float fb0, dfb, fz0, dfz, t0, dt, L;
  int i0, i1;  // inclusive sample range that may carry non-zero weight
};

__device__ __forceinline__ void clip_range(float f0, float df, float lo_b, float hi_b, float &lo,
                                           float &hi) {
  if (fabsf(df) < 1e-20f) {
    if (!(f0 > lo_b && f0 < hi_b)) { lo = 1e30f; hi = -1e30f; }
    return;
  }
  float t1 = (lo_b - f0) / df, t2 = (hi_b - f0) / df;
  lo = fmaxf(lo, fminf(t1, t2));
  hi = fminf(hi, fmaxf(t1, t2));
}

__device__ __forceinline__ void lor_setup(const DevPlan &P, int v, int p, int r, Lor &L) {
  const float4 vw = __ldg(&P.view[v]);
  const float4 vr = __ldg(&P.vr[v * P.nrad + r]);
  const float4 pl = __ldg(&P.plane[p]);
  L.xdrive = vw.x != 0.f;
  L.dfb = vw.y;
  const float dau = vw.z;
  L.fb0 = vr.x;
  const float t0b = vr.y, inv2h = vr.z;
  const float g1 = dau * inv2h, g2 = t0b * inv2h;
  L.dfz = g1 * pl.y;
  L.fz0 = fmaf(g2, pl.y, pl.x);
  const float k = pl.z * inv2h;
  const float sec = sqrtf(fmaf(k, k, 1.f));
  L.L = fabsf(dau) * sec;
  L.t0 = t0b * sec;
  L.dt = dau * sec;
  const int Na = L.xdrive ? P.nx : P.ny;
  const int Nb = L.xdrive ? P.ny : P.nx;
  float lo = 0.f, hi = (float)(Na - 1);
  clip_range(L.fb0, L.dfb, -1.f, (float)Nb, lo, hi);
  clip_range(L.fz0, L.dfz, -1.f, (float)P.nz, lo, hi);
  if (lo > hi) { L.i0 = 1; L.i1 = 0; return; }
  lo = fmaxf(lo, -2.f);
  hi = fminf(hi, (float)Na + 1.f);
  L.i0 = max(0, (int)floorf(lo) - 1);
  L.i1 = min(Na - 1, (int)ceilf(hi) + 1);
}

// Makes the sample range uniform across the warp (union of the lanes' ranges) so that
// at every step all lanes sample the same driving plane and touch adjacent voxels.
// Samples outside a lane's own range fall outside the image and carry zero weight, so
// the sums are unchanged.  Every lane of the warp must call this.
__device__ __forceinline__ void warp_uniform_range(Lor &L, bool valid) {
  const bool own = valid && L.i0 <= L.i1;
  const int lo = __reduce_min_sync(0xffffffffu, own ? L.i0 : 0x7fffffff);
  const int hi = __reduce_max_sync(0xffffffffu, own ? L.i1 : -1);
  // an empty union becomes [0, -1]: loops start at i0 + part and must not overflow
  L.i0 = lo <= hi ? lo : 0;
  L.i1 = lo <= hi ? hi : -1;
}

// Bilinear sample position at plane i.
struct Samp {
  int base;       // frame index of neighbour (iz, i, ib)
  float wb, wz;   // fractional parts
  bool b0, b1, z0, z1;
};

__device__ __forceinline__ void sample_at(const Lor &L, int i, int Na, int Nb, int Nz, Samp &S) {
  const float fb = fmaf((float)i, L.dfb, L.fb0);
  const float fz = fmaf((float)i, L.dfz, L.fz0);
  const float fbf = floorf(fb), fzf = floorf(fz);
  const int ib = (int)fbf, iz = (int)fzf;
  S.wb = fb - fbf;
  S.wz = fz - fzf;
  // neighbours outside the image, or with an exactly-zero weight (e.g. the upper row of
  // a direct plane, whose axial coordinate is an exact slice index), are skipped
  S.b0 = (unsigned)ib < (unsigned)Nb;
  S.b1 = (unsigned)(ib + 1) < (unsigned)Nb && S.wb != 0.f;
  S.z0 = (unsigned)iz < (unsigned)Nz;
  S.z1 = (unsigned)(iz + 1) < (unsigned)Nz && S.wz != 0.f;
  S.base = (iz * Na + i) * Nb + ib;
}

// G(u) = erfc(|clamp(u)|) at one TOF bin edge; the truncated-Gaussian bin weight
// between edges lo < hi is (erf(clamp(u_hi)) - erf(clamp(u_lo))) / (2 erf(amax)),
// evaluated from G in the form that avoids cancellation in the tails.
__device__ __forceinline__ float tof_edge_G(const DevPlan &P, const float *tab, float u) {
  const float au = fabsf(u);
  if (!(au < P.tof_amax)) return P.tof_erfc_amax;
  const float xs = au * P.erfc_scale;
  const int j = min((int)xs, kErfcTab - 1);
  const float f = xs - (float)j;
  const float a = tab[j];
  return fmaf(f, tab[j + 1] - a, a);
}

// Copies the erfc table into shared memory (every thread of the block must call this).
__device__ __forceinline__ void load_erfc_tab(const DevPlan &P, float *s_tab) {
  for (int k = threadIdx.x + blockDim.x * threadIdx.y; k <= kErfcTab; k += blockDim.x * blockDim.y)
    s_tab[k] = __ldg(&P.erfc_tab[k]);
  __syncthreads();
}

__device__ __forceinline__ float tof_bin_weight(const DevPlan &P, float ulo, float Glo, float uhi,
                                                float Ghi) {
  float w;
  if (ulo >= 0.f) w = Glo - Ghi;
  else if (uhi < 0.f) w = Ghi - Glo;
  else w = (2.f - Glo) - Ghi;
  return w * P.tof_half_norm;
}

// Counts y as float.
__device__ __forceinline__ float load_y(const DevPlan &P, size_t idx) {
  if (P.yt == PET_Y_U16) return (float)__ldg(((const uint16_t *)P.y) + idx);
  if (P.yt == PET_Y_U32) return (float)__ldg(((const uint32_t *)P.y) + idx);
  return __ldg(((const float *)P.y) + idx);
}

// ----------------------------------------------------------------- launchers
// Count of kernel launches enqueued by this library (graph replays add the number of
// kernel nodes of the replayed graph).
void note_launch(long long n = 1);
long long launch_count();

// Projector kernels (proj_kernels.cu).  `subset` < 0 means all views.
enum GradMode { MODE_GRAD = 0, MODE_EM = 1, MODE_OBJ = 2, MODE_SENS = 3, MODE_NGRAD = 4 };
// MODE_NGRAD backprojects -q: added to a MODE_GRAD result at another image it forms the
// difference of two subset gradients (low-memory SVRG).
__host__ __device__ __forceinline__ bool grad_like(int mode) { return mode == MODE_GRAD || mode == MODE_NGRAD; }

cudaError_t launch_forward(const DevPlan &P, int subset, const float *x, const float *xT,
                           float *out, cudaStream_t st);
cudaError_t launch_back(const DevPlan &P, int subset, const float *q, float *g, float *gT,
                        cudaStream_t st);
cudaError_t launch_back_det(const DevPlan &P, const DevPlanDet &D, int subset, const float *q,
                            float *g, int ones, cudaStream_t st);
int ratio_blocks(const DevPlan &P, int subset);
cudaError_t launch_ratio(const DevPlan &P, int subset, const float *ax, float *q, double *kl_part,
                         int mode, cudaStream_t st);
// Fused forward -> ratio -> back over one subset (or all views).  mode MODE_GRAD:
// q = m (1 - y/ybar); MODE_EM: q = m y/ybar; MODE_OBJ: no backprojection; MODE_SENS:
// q = m (backprojects ones).  kl_part: per-block FP64 partial sums of the KL term
// (may be NULL).  subset_dev (may be NULL) overrides `subset` from device memory.
cudaError_t launch_grad(const DevPlan &P, int subset, const int *subset_dev, const float *x,
                        const float *xT, float *g, float *gT, double *kl_part, int mode,
                        int *nblocks_out, cudaStream_t st);
int grad_blocks(const DevPlan &P, int max_views);
// Largest parts per LOR (16 without TOF, 8 with the windowed TOF kernel, else 4) and
// planes per thread (4 without TOF or with the windowed TOF kernel, else 1) of the fused
// gradient for this plan.
int max_split(const DevPlan &P);
int max_planes(const DevPlan &P);
cudaError_t launch_fill(float *p, size_t n, float v, cudaStream_t st);

// Subset index that marks an instance of a batch as skipped for one batched iteration
// (it runs that window alone).
constexpr int kBatchSkip = -2;

// One reconstruction of a batch, as seen by the batched fused-gradient kernel.
struct GradJob {
  DevPlan P;
  const int *subset_dev;  // this job's subset for the iteration
  const float *x, *xT;
  float *g, *gT;
};
// Blocks [begin[j], begin[j+1]) belong to job j; all jobs use one launch shape (K, split).
cudaError_t launch_grad_batch(const GradJob *jobs, const int *begin, int njobs, int total_blocks, int K,
                              int split, cudaStream_t st);
int grad_blocks_shape(const DevPlan &P, int nv, int K, int split);
// Windowed TOF fused gradient (tof_kernels.cu): usable for this plan with K planes per
// thread (1, 2 or 4)?  Blocks of a launch over nv views, and the launch itself.
bool tofk_supported(const DevPlan &P, int K);
// Sets the dynamic shared-memory limits of the windowed TOF kernels on the current device
// (called when a plan that uses them is created, outside any stream capture).
cudaError_t tofk_init_device();
int tofk_blocks(const DevPlan &P, int nv, int K, int split);
cudaError_t launch_grad_tofk(const DevPlan &P, int K, int split, unsigned grid, int subset, const int *subset_dev,
                             const float *x, const float *xT, float *g, float *gT, double *kl_part, int mode,
                             cudaStream_t st);
cudaError_t launch_transpose(const float *src, float *dst, int nx, int ny, int nz, int to_xfast,
                             int accumulate, cudaStream_t st);
cudaError_t launch_mult(const DevPlan &P, const float *mu, const float *muT, const float *sens,
                        float *m, cudaStream_t st);

// Image kernels (image_kernels.cu).
// Image-space resolution model: taps w[k + R], |k| <= R, of one axis (R = 0: identity).
constexpr int kGaussMaxR = 31;
struct GaussTaps {
  int R;
  float w[2 * kGaussMaxR + 1];
};
// out = G in with the per-axis taps t[0..2] (x, y, z; the z pass is skipped when nz = 1);
// tmp is an image-sized scratch distinct from in and out (in and out may alias).
cudaError_t launch_gauss(const GaussTaps *t, int nx, int ny, int nz, const float *in, float *out, float *tmp,
                         cudaStream_t st);

struct RdpArgs {
  int nx, ny, nz;
  float w[7];  // weights for offsets (1,0,0),(0,1,0),(0,0,1),(1,1,0),(1,0,1),(0,1,1),(1,1,1)
  float gamma, eps, scale;
  const float *kappa;
  int zch;  // slices per stencil block: 2, 4 or 8
};
constexpr int kRdpZchDefault = 4;
// The slice count a stencil launch uses: 2, 4 or 8 (anything else falls back to 4), so
// that the block count and the kernel's shared-memory planes always agree.
__host__ __device__ __forceinline__ int rdp_zch_valid(int zch) {
  return (zch == 2 || zch == 4 || zch == 8) ? zch : kRdpZchDefault;
}
RdpArgs make_rdp_args(const pet_rdp_params &p);
cudaError_t launch_rdp(const RdpArgs &a, const float *x, float *grad, float *hdiag,
                       double *val_part, int accumulate, int *nblocks_out, cudaStream_t st);
// Stencil blocks of an image with zch slices per block (the default tile unless given).
int rdp_blocks(int nx, int ny, int nz, int zch = kRdpZchDefault);
struct RdpJob {
  RdpArgs a;
  const float *x;
  float *grad;
};
// sub (may be NULL): per-job subsets of the iteration; jobs marked kBatchSkip are skipped.
cudaError_t launch_rdp_batch(const RdpJob *jobs, const int *begin, int njobs, int total_blocks,
                             const int *sub, cudaStream_t st);
cudaError_t launch_reduce_sum(const double *part, int n, double *out, int accumulate,
                              cudaStream_t st);
cudaError_t launch_max(const float *x, size_t n, float *part, float *out, cudaStream_t st);
int max_blocks(size_t n);
cudaError_t launch_precond(const float *x, const float *sens, const float *hdiag, float alpha,
                           const float *xmax, float delta_rel, float *D, size_t n,
                           cudaStream_t st);
cudaError_t launch_em_apply(float *x, const float *bp, const float *sens, size_t n,
                            cudaStream_t st);
cudaError_t launch_nrmse(const float *x, const float *ref, const uint8_t *mask, const uint8_t *bg,
                         size_t n, double *part, double *out, cudaStream_t st);
int nrmse_blocks(size_t n);

}  // namespace petgb
