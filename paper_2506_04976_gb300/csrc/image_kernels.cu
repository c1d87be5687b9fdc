// Image-domain kernels for sm_103a: the 26-neighbour relative difference prior
// (eq. 3; gradient and Hessian diagonal of Appendix A.1) as a 3D stencil with halo
// tiles in shared memory, deterministic FP64 reductions, the diagonal preconditioners
// of Sec. 2.3 (eq. 8), the EM update and the NRMSE of Sec. 3.1.
#include <math.h>

#include <algorithm>

#include "pet_internal.cuh"

namespace petgb {

// tile: 32 x 8 voxels x zch slices (zch = 2, 4 or 8, chosen per image by the autotuners;
// default 4); the shared-memory planes are sized for the largest
constexpr int RDP_TX = 32, RDP_TY = 8, RDP_ZMAX = 8;

RdpArgs make_rdp_args(const pet_rdp_params &p) {
  RdpArgs a;
  a.nx = p.nx; a.ny = p.ny; a.nz = p.nz;
  const double dmin = fmin(p.dx, fmin(p.dy, p.dz));
  const int off[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
  for (int k = 0; k < 7; ++k) {
    const double ex = off[k][0] * p.dx, ey = off[k][1] * p.dy, ez = off[k][2] * p.dz;
    a.w[k] = (float)(dmin / sqrt(ex * ex + ey * ey + ez * ez));
  }
  a.gamma = p.gamma; a.eps = p.eps; a.scale = p.scale; a.kappa = p.kappa;
  a.zch = kRdpZchDefault;
  return a;
}

int rdp_blocks(int nx, int ny, int nz, int zch) {
  zch = rdp_zch_valid(zch);
  return ((nx + RDP_TX - 1) / RDP_TX) * ((ny + RDP_TY - 1) / RDP_TY) * ((nz + zch - 1) / zch);
}

__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double red[32];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthreads = blockDim.x * blockDim.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (tid < 32) {
    s = tid < (nthreads >> 5) ? red[tid] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// Per-voxel RDP sums over the 26 neighbours held in the shared-memory planes (plane
// index lz = local z + 1).  BOUND enables the image-boundary checks.
template <bool KAPPA, bool WG, bool WH, bool VAL, bool BOUND>
__device__ __forceinline__ void rdp_voxel(const RdpArgs &a, const float (*sx)[RDP_TY + 2][RDP_TX + 2],
                                          const float (*sk)[RDP_TY + 2][RDP_TX + 2], int z, int lz, int gx,
                                          int gy, int tx, int ty, float &gsum, float &hsum, float &vs) {
  const float xi = sx[lz][ty + 1][tx + 1];
  const float ki = KAPPA ? sk[lz][ty + 1][tx + 1] : 1.f;
#pragma unroll
  for (int oz = -1; oz <= 1; ++oz) {
    if (BOUND && (z + oz < 0 || z + oz >= a.nz)) continue;
    const int sl = lz + oz;
#pragma unroll
    for (int oy = -1; oy <= 1; ++oy) {
      if (BOUND && (gy + oy < 0 || gy + oy >= a.ny)) continue;
#pragma unroll
      for (int ox = -1; ox <= 1; ++ox) {
        if (ox == 0 && oy == 0 && oz == 0) continue;
        if (BOUND && (gx + ox < 0 || gx + ox >= a.nx)) continue;
        constexpr int widx[8] = {-1, 0, 1, 3, 2, 4, 5, 6};
        const int code = (ox != 0 ? 1 : 0) + (oy != 0 ? 2 : 0) + (oz != 0 ? 4 : 0);
        float w = a.w[widx[code]];
        const float xj = sx[sl][ty + 1 + oy][tx + 1 + ox];
        if (KAPPA) w *= ki * sk[sl][ty + 1 + oy][tx + 1 + ox];
        const float d = xi - xj;
        const float ad = fabsf(d);
        const float phi = (xi + xj) + a.gamma * ad + a.eps;
        const float inv = __fdividef(1.f, phi);
        const float inv2 = inv * inv;
        if (WG) gsum = fmaf(w * d * ((2.f * phi - d) - a.gamma * ad), inv2, gsum);
        if (WH) {
          const float e2 = fmaf(2.f, xj, a.eps);
          hsum = fmaf(2.f * w * e2 * e2, inv2 * inv, hsum);
        }
        if (VAL) vs = fmaf(w * d * d, inv, vs);
      }
    }
  }
}

// One block: a 32x8 tile over a.zch slices.  All zch + 2 planes (with halo) are staged in
// shared memory at once, then every slice is computed without further barriers.
template <bool KAPPA, bool WG, bool WH, bool VAL>
__device__ __forceinline__ void rdp_body(const RdpArgs &a, const float *__restrict__ x, float *__restrict__ grad,
                                         float *__restrict__ hdiag, double *__restrict__ val_out, int accumulate,
                                         int blk) {
  __shared__ float sx[RDP_ZMAX + 2][RDP_TY + 2][RDP_TX + 2];
  __shared__ float sk[KAPPA ? RDP_ZMAX + 2 : 1][RDP_TY + 2][RDP_TX + 2];
  const int zch = rdp_zch_valid(a.zch);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RDP_TX + tx;
  const int nbx = (a.nx + RDP_TX - 1) / RDP_TX, nby = (a.ny + RDP_TY - 1) / RDP_TY;
  const int bx = blk % nbx, by = (blk / nbx) % nby, bz = blk / (nbx * nby);
  const int x0 = bx * RDP_TX, y0 = by * RDP_TY;
  const int z0 = bz * zch, z1 = min(a.nz, z0 + zch);
  const int nxy = a.nx * a.ny;
  const bool inner_xy = x0 >= 1 && x0 + RDP_TX < a.nx && y0 >= 1 && y0 + RDP_TY < a.ny;
  constexpr int PLANE = (RDP_TY + 2) * (RDP_TX + 2);
  for (int e = tid; e < (zch + 2) * PLANE; e += RDP_TX * RDP_TY) {
    const int lz = e / PLANE, rem = e % PLANE;
    const int ly = rem / (RDP_TX + 2), lx = rem % (RDP_TX + 2);
    const int z = z0 + lz - 1, gx = x0 + lx - 1, gy = y0 + ly - 1;
    float v = 0.f, kv = 0.f;
    if (z >= 0 && z < a.nz && gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny) {
      const size_t gi = (size_t)z * nxy + (size_t)gy * a.nx + gx;
      v = __ldg(x + gi);
      if (KAPPA) kv = __ldg(a.kappa + gi);
    }
    sx[lz][ly][lx] = v;
    if (KAPPA) sk[lz][ly][lx] = kv;
  }
  __syncthreads();
  double vsum = 0.0;
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx < a.nx && gy < a.ny) {
    for (int z = z0; z < z1; ++z) {
      const int lz = z - z0 + 1;
      float gsum = 0.f, hsum = 0.f, vs = 0.f;
      if (inner_xy && z >= 1 && z + 1 < a.nz)
        rdp_voxel<KAPPA, WG, WH, VAL, false>(a, sx, sk, z, lz, gx, gy, tx, ty, gsum, hsum, vs);
      else
        rdp_voxel<KAPPA, WG, WH, VAL, true>(a, sx, sk, z, lz, gx, gy, tx, ty, gsum, hsum, vs);
      const size_t gi = (size_t)z * nxy + (size_t)gy * a.nx + gx;
      if (WG) grad[gi] = accumulate ? fmaf(a.scale, gsum, grad[gi]) : a.scale * gsum;
      if (WH) hdiag[gi] = a.scale * hsum;
      if (VAL) vsum += 0.5 * (double)vs;
    }
  }
  if (VAL) {
    const double s = block_sum_d(vsum * (double)a.scale);
    if (tid == 0) *val_out = s;
  }
}

template <bool KAPPA, bool WG, bool WH, bool VAL>
__global__ void __launch_bounds__(RDP_TX * RDP_TY) k_rdp(RdpArgs a, const float *__restrict__ x,
                                                          float *__restrict__ grad, float *__restrict__ hdiag,
                                                          double *__restrict__ val_part, int accumulate) {
  rdp_body<KAPPA, WG, WH, VAL>(a, x, grad, hdiag, VAL ? val_part + blockIdx.x : nullptr, accumulate, blockIdx.x);
}

// Batched RDP gradient (no kappa, gradient only): blocks [begin[j], begin[j+1]) belong
// to job j.
__global__ void __launch_bounds__(RDP_TX * RDP_TY) k_rdp_batch(const RdpJob *__restrict__ jobs,
                                                                const int *__restrict__ begin, int njobs,
                                                                const int *__restrict__ sub) {
  __shared__ int s_job;
  __shared__ RdpJob sj;
  const int tid = threadIdx.y * RDP_TX + threadIdx.x;
  if (tid < 32) {
    int job = 0;
    for (int base = 0; base < njobs; base += 32) {
      const int j = base + tid;
      const unsigned m = __ballot_sync(0xffffffffu, j < njobs && __ldg(&begin[j]) <= (int)blockIdx.x);
      job = base + __popc(m) - 1;
      if (m != 0xffffffffu) break;
    }
    if (tid == 0) { s_job = job; sj = jobs[job]; }
  }
  __syncthreads();
  if (sub && __ldg(&sub[s_job]) == kBatchSkip) return;  // whole block: one job
  const int blk = (int)blockIdx.x - __ldg(&begin[s_job]);
  if (sj.a.kappa)  // block-uniform: the job's kappa-weighted prior
    rdp_body<true, true, false, false>(sj.a, sj.x, sj.grad, nullptr, nullptr, 0, blk);
  else
    rdp_body<false, true, false, false>(sj.a, sj.x, sj.grad, nullptr, nullptr, 0, blk);
}

cudaError_t launch_rdp_batch(const RdpJob *jobs, const int *begin, int njobs, int total_blocks,
                             const int *sub, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  note_launch();
  k_rdp_batch<<<total_blocks, dim3(RDP_TX, RDP_TY), 0, st>>>(jobs, begin, njobs, sub);
  return cudaGetLastError();
}

template <bool KAPPA>
static void rdp_dispatch(const RdpArgs &a, int nb, dim3 block, const float *x, float *grad, float *hdiag,
                         double *val_part, int accumulate, cudaStream_t st) {
  const int code = (grad ? 1 : 0) | (hdiag ? 2 : 0) | (val_part ? 4 : 0);
  switch (code) {
    case 1: k_rdp<KAPPA, true, false, false><<<nb, block, 0, st>>>(a, x, grad, hdiag, val_part, accumulate); break;
    case 2: k_rdp<KAPPA, false, true, false><<<nb, block, 0, st>>>(a, x, grad, hdiag, val_part, accumulate); break;
    case 3: k_rdp<KAPPA, true, true, false><<<nb, block, 0, st>>>(a, x, grad, hdiag, val_part, accumulate); break;
    case 4: k_rdp<KAPPA, false, false, true><<<nb, block, 0, st>>>(a, x, grad, hdiag, val_part, accumulate); break;
    case 5: k_rdp<KAPPA, true, false, true><<<nb, block, 0, st>>>(a, x, grad, hdiag, val_part, accumulate); break;
    case 6: k_rdp<KAPPA, false, true, true><<<nb, block, 0, st>>>(a, x, grad, hdiag, val_part, accumulate); break;
    case 7: k_rdp<KAPPA, true, true, true><<<nb, block, 0, st>>>(a, x, grad, hdiag, val_part, accumulate); break;
    default: break;
  }
}

cudaError_t launch_rdp(const RdpArgs &a, const float *x, float *grad, float *hdiag,
                       double *val_part, int accumulate, int *nblocks_out, cudaStream_t st) {
  const int nb = rdp_blocks(a.nx, a.ny, a.nz, a.zch);
  if (nblocks_out) *nblocks_out = nb;
  if (!grad && !hdiag && !val_part) return cudaSuccess;
  dim3 block(RDP_TX, RDP_TY);
  note_launch();
  if (a.kappa) rdp_dispatch<true>(a, nb, block, x, grad, hdiag, val_part, accumulate, st);
  else rdp_dispatch<false>(a, nb, block, x, grad, hdiag, val_part, accumulate, st);
  return cudaGetLastError();
}

// Deterministic sum of n partials: fixed strided order per thread, fixed tree.
__global__ void k_reduce_sum(const double *__restrict__ part, int n, double *out, int accumulate) {
  __shared__ double s[1024];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = accumulate ? *out + s[0] : s[0];
}

cudaError_t launch_reduce_sum(const double *part, int n, double *out, int accumulate,
                              cudaStream_t st) {
  note_launch();
  k_reduce_sum<<<1, 1024, 0, st>>>(part, n, out, accumulate);
  return cudaGetLastError();
}

int max_blocks(size_t n) { return (int)min((size_t)1024, (n + 1023) / 1024); }

__global__ void k_max_part(const float *__restrict__ x, size_t n, float *part) {
  __shared__ float s[256];
  float m = -INFINITY;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, x[i]);
  s[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] = fmaxf(s[threadIdx.x], s[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_max_final(const float *part, int n, float *out) {
  __shared__ float s[1024];
  float m = -INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, part[i]);
  s[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] = fmaxf(s[threadIdx.x], s[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

cudaError_t launch_max(const float *x, size_t n, float *part, float *out, cudaStream_t st) {
  const int nb = max_blocks(n);
  note_launch();
  k_max_part<<<nb, 256, 0, st>>>(x, n, part);
  note_launch();
  k_max_final<<<1, 1024, 0, st>>>(part, nb, out);
  return cudaGetLastError();
}

// D = (x+delta)/(sens + alpha h (x+delta)), delta = delta_rel * max(x); h == NULL: MLEM.
__global__ void k_precond(const float *__restrict__ x, const float *__restrict__ sens,
                          const float *__restrict__ h, float alpha, const float *xmax, float delta_rel,
                          float *__restrict__ D, size_t n) {
  const float delta = delta_rel * fmaxf(*xmax, 0.f);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float num = x[i] + delta;
    float den = sens[i];
    if (h) den = fmaf(alpha * h[i], num, den);
    D[i] = den > 0.f ? num / den : 0.f;
  }
}

static unsigned grid_1d(size_t n) { return (unsigned)min((size_t)152 * 16, (n + 255) / 256); }

cudaError_t launch_precond(const float *x, const float *sens, const float *hdiag, float alpha,
                           const float *xmax, float delta_rel, float *D, size_t n,
                           cudaStream_t st) {
  note_launch();
  k_precond<<<grid_1d(n), 256, 0, st>>>(x, sens, hdiag, alpha, xmax, delta_rel, D, n);
  return cudaGetLastError();
}

__global__ void k_em_apply(float *__restrict__ x, const float *__restrict__ bp,
                           const float *__restrict__ sens, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float s = sens[i];
    if (s > 0.f) x[i] = x[i] / s * bp[i];
  }
}

cudaError_t launch_em_apply(float *x, const float *bp, const float *sens, size_t n,
                            cudaStream_t st) {
  note_launch();
  k_em_apply<<<grid_1d(n), 256, 0, st>>>(x, bp, sens, n);
  return cudaGetLastError();
}

int nrmse_blocks(size_t n) { return (int)min((size_t)1024, (n + 1023) / 1024); }

__global__ void k_nrmse_part(const float *__restrict__ x, const float *__restrict__ ref,
                             const uint8_t *__restrict__ mask, const uint8_t *__restrict__ bg, size_t n,
                             double *part) {
  double se = 0, nm = 0, sb = 0, nb = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (mask[i]) { const double d = (double)x[i] - (double)ref[i]; se += d * d; nm += 1; }
    if (bg[i]) { sb += ref[i]; nb += 1; }
  }
  double r;
  r = block_sum_d(se); if (threadIdx.x == 0) part[4 * blockIdx.x + 0] = r;
  r = block_sum_d(nm); if (threadIdx.x == 0) part[4 * blockIdx.x + 1] = r;
  r = block_sum_d(sb); if (threadIdx.x == 0) part[4 * blockIdx.x + 2] = r;
  r = block_sum_d(nb); if (threadIdx.x == 0) part[4 * blockIdx.x + 3] = r;
}

__global__ void k_nrmse_final(const double *part, int nb, double *out) {
  if (threadIdx.x != 0) return;
  double se = 0, nm = 0, sb = 0, nbg = 0;
  for (int b = 0; b < nb; ++b) {
    se += part[4 * b]; nm += part[4 * b + 1]; sb += part[4 * b + 2]; nbg += part[4 * b + 3];
  }
  *out = sqrt(se / nm) / (sb / nbg);
}

cudaError_t launch_nrmse(const float *x, const float *ref, const uint8_t *mask, const uint8_t *bg,
                         size_t n, double *part, double *out, cudaStream_t st) {
  const int nb = nrmse_blocks(n);
  note_launch();
  k_nrmse_part<<<nb, 256, 0, st>>>(x, ref, mask, bg, n, part);
  note_launch();
  k_nrmse_final<<<1, 32, 0, st>>>(part, nb, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------ resolution model
// One separable pass of the image-space Gaussian along axis AXIS (0 x, 1 y, 2 z):
// out[i] = sum_k w[k + R] in[i + k e_AXIS], neighbours outside the image omitted.
// One thread per output voxel; consecutive threads take consecutive x, so every tap
// is a coalesced row read (the image is L2-resident at the sizes of interest).
template <int AXIS>
__global__ void __launch_bounds__(256) k_gauss(const float *__restrict__ in, float *__restrict__ out, int nx,
                                              int ny, int nz, GaussTaps t) {
  const size_t N = (size_t)nx * ny * nz;
  const int n = AXIS == 0 ? nx : AXIS == 1 ? ny : nz;
  const size_t stride = AXIS == 0 ? 1 : AXIS == 1 ? (size_t)nx : (size_t)nx * ny;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const int c = AXIS == 0 ? (int)(i % nx) : AXIS == 1 ? (int)((i / nx) % ny) : (int)(i / ((size_t)nx * ny));
    const int k0 = max(-t.R, -c), k1 = min(t.R, n - 1 - c);
    float acc = 0.f;
    for (int k = k0; k <= k1; ++k) acc = fmaf(t.w[k + t.R], __ldg(in + (long long)i + (long long)k * (long long)stride), acc);
    out[i] = acc;
  }
}

cudaError_t launch_gauss(const GaussTaps *t, int nx, int ny, int nz, const float *in, float *out, float *tmp,
                         cudaStream_t st) {
  const size_t N = (size_t)nx * ny * nz;
  const unsigned grid = (unsigned)std::min<size_t>((size_t)152 * 8, (N + 255) / 256);
  note_launch();
  k_gauss<0><<<grid, 256, 0, st>>>(in, tmp, nx, ny, nz, t[0]);
  note_launch();
  k_gauss<1><<<grid, 256, 0, st>>>(tmp, out, nx, ny, nz, t[1]);
  if (nz > 1) {
    note_launch();
    k_gauss<2><<<grid, 256, 0, st>>>(out, tmp, nx, ny, nz, t[2]);
    cudaError_t e = cudaMemcpyAsync(out, tmp, N * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace petgb
