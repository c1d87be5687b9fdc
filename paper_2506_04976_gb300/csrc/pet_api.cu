// Host side of the C ABI declared in include/pet_gb300.h: plan construction (geometry
// tables in the driving frame of each view), data binding (attenuation factors and
// sensitivity images), and the operator entry points.  Every entry point validates its
// arguments on the host, enqueues kernels on the caller's stream and returns a status.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pet_internal.cuh"
#include "pet_plan.h"

using namespace petgb;

#define PET_CK(call)                                  \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return PET_ERR_CUDA;       \
  } while (0)

extern "C" const char *pet_status_str(pet_status st) {
  switch (st) {
    case PET_OK: return "ok";
    case PET_ERR_ARG: return "invalid argument";
    case PET_ERR_SHAPE: return "geometry not representable";
    case PET_ERR_INFEASIBLE: return "infeasible data: ybar <= 0 where y > 0";
    case PET_ERR_TIMEOUT: return "bounded device wait timed out";
    case PET_ERR_CUDA: return "CUDA runtime error";
    case PET_ERR_UNSUPPORTED: return "unsupported configuration";
    case PET_ERR_STATE: return "invalid call order";
    case PET_ERR_NOMEM: return "device allocation failed";
  }
  return "unknown status";
}

static cudaStream_t S(void *st) { return (cudaStream_t)st; }

template <class T>
static cudaError_t dalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMalloc((void **)p, count * sizeof(T));
}

// Driving axis of view v: x when |u_x|/dx >= |u_y|/dy, u = (-sin phi, cos phi).  For
// square pixels the comparison is the exact integer test V <= 4v <= 3V.
static int view_xdrive(const pet_geometry &g, int v) {
  if (g.dx == g.dy) return (4 * v >= g.nview && 4 * v <= 3 * g.nview) ? 1 : 0;
  const double phi = v * M_PI / g.nview;
  return fabs(sin(phi)) * g.dy >= fabs(cos(phi)) * g.dx ? 1 : 0;
}

static void plan_free(pet_plan *p) {
  if (!p) return;
  cudaFree(p->d_view); cudaFree(p->d_vr); cudaFree(p->d_plane); cudaFree(p->d_aff);
  cudaFree(p->d_m); cudaFree(p->d_sens); cudaFree(p->d_sens_sub);
  cudaFree(p->d_xT); cudaFree(p->d_gT); cudaFree(p->d_part); cudaFree(p->d_err);
  cudaFree(p->d_fpart); cudaFree(p->d_fscalar); cudaFree(p->d_qtmp); cudaFree(p->d_img);
  cudaFree(p->d_groups); cudaFree(p->d_gzd); cudaFree(p->d_gplane); cudaFree(p->d_gzs);
  cudaFree(p->d_erfc_tab);
  cudaFree(p->d_tofw_tab);
  cudaFree(p->d_tof_grp2);
  cudaFree(p->d_tof_grp4);
  cudaFree(p->d_tof_work);
  cudaFree(p->d_tof_xp);
  cudaFree(p->d_tof_xtp);
  cudaFree(p->d_tof_gp);
  cudaFree(p->d_tof_gtp);
  cudaFree(p->d_xs); cudaFree(p->d_rtmp);
  delete p;
}

// Taps of the resolution model along one axis of spacing delta: the Gaussian of the
// given FWHM sampled at k delta, |k| <= ceil(3 sigma / delta), normalised to unit sum.
static bool gauss_taps(double fwhm, double delta, GaussTaps &t) {
  const double sigma = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
  const double Rd = ceil(3.0 * sigma / delta);
  if (!(Rd <= kGaussMaxR)) return false;
  t.R = (int)Rd;
  double w[2 * kGaussMaxR + 1], sum = 0.0;
  for (int k = -t.R; k <= t.R; ++k) {
    w[k + t.R] = exp(-(k * delta) * (k * delta) / (2.0 * sigma * sigma));
    sum += w[k + t.R];
  }
  for (int k = 0; k < 2 * kGaussMaxR + 1; ++k) t.w[k] = k <= 2 * t.R ? (float)(w[k] / sum) : 0.f;
  return true;
}

// Truncated-Gaussian TOF weight of a sample at signed distance d from a bin centre: the
// mass of N(0, sigma^2) truncated to +-3 sigma (renormalised) inside [d - w/2, d + w/2].
static double tof_F(double d, double sigma, double w) {
  const double amax = 3.0 / sqrt(2.0);
  double uhi = (0.5 * w - d) / (sqrt(2.0) * sigma), ulo = (-0.5 * w - d) / (sqrt(2.0) * sigma);
  uhi = std::min(amax, std::max(-amax, uhi));
  ulo = std::min(amax, std::max(-amax, ulo));
  return (erf(uhi) - erf(ulo)) / (2.0 * erf(amax));
}

// Tables of the windowed TOF kernel: F sampled at nodes -R + k h (h = w / kTofM, R =
// 3 sigma + w/2, k = 0..Ktab with Ktab = ceil(2R/h)), stored by window rows: for a sample
// whose node index for its lowest bin is ib = row + Ktab - kTofM, window bin j has node
// n_j = ib - j M, value F(n_j) and slope F(n_j + 1) - F(n_j); a row holds the bins in
// pairs (F_2p, F_2p+1, slope_2p, slope_2p+1), padded to the kernel's even WIN (4, 6 or
// 8).  Also the groups of 2 and 4 consecutive planes with equal axial slope (the planes
// of a thread share their TOF weights).
static pet_status build_tof_window(pet_plan *pl, const std::vector<float4> &plane) {
  const pet_geometry &g = pl->g;
  DevPlan &dp = pl->dp;
  const double w = g.tof_bin, sigma = g.tof_sigma;
  const double R = 3.0 * sigma + 0.5 * w, h = w / kTofM;
  const long long Ktab = (long long)ceil(2.0 * R / h);
  const int win = (int)((Ktab - 1) / kTofM) + 1;
  dp.tofw_win = win;
  if (win > 8) return PET_OK;  // too many bins per sample for the register window
  const int wk = win <= 4 ? 4 : (win <= 6 ? 6 : 8);
  const double c0 = -0.5 * (pl->T - 1) * w;
  dp.tofw_inv_h = (float)(1.0 / h);
  dp.tofw_off = (float)((R - c0) / h - (double)Ktab + kTofM);
  std::vector<float4> tab((size_t)kTofM * (wk / 2));
  for (int row = 0; row < kTofM; ++row) {
    const long long ib = row + Ktab - kTofM;
    float fv[8], fs[8];
    for (int j = 0; j < wk; ++j) {
      const long long kn = ib - (long long)j * kTofM;
      const double a = tof_F(-R + kn * h, sigma, w), b = tof_F(-R + (kn + 1) * h, sigma, w);
      fv[j] = (float)a;
      fs[j] = (float)(b - a);
    }
    for (int q = 0; q < wk / 2; ++q)
      tab[(size_t)row * (wk / 2) + q] = make_float4(fv[2 * q], fv[2 * q + 1], fs[2 * q], fs[2 * q + 1]);
  }
  // groups of up to K consecutive planes of equal axial slope, padded with -1
  const int P = g.nplane;
  auto groups = [&](int K) {
    std::vector<int> grp;
    for (int p = 0; p < P;) {
      int c = 1;
      while (c < K && p + c < P && plane[p + c].z == plane[p].z) ++c;
      for (int k = 0; k < K; ++k) grp.push_back(k < c ? p + k : -1);
      p += c;
    }
    return grp;
  };
  const std::vector<int> grp2 = groups(2), grp4 = groups(4);
  // whether the planes of every group lie a whole number of slices apart (their axial
  // positions then share one fraction along the LOR)
  auto zs = [&](int p) { return (g.z1[p] + g.z2[p]) / (2.0 * g.dz); };
  auto whole = [&](const std::vector<int> &grp, int K) {
    for (size_t q = 0; q < grp.size(); q += K)
      for (int k = 1; k < K; ++k) {
        if (grp[q + k] < 0) continue;
        const double d = zs(grp[q + k]) - zs(grp[q]);
        if (fabs(d - nearbyint(d)) > 1e-9) return false;
      }
    return true;
  };
  dp.tof_zint = whole(grp2, 2) && whole(grp4, 4) ? 1 : 0;
  if (dalloc(&pl->d_tofw_tab, tab.size()) != cudaSuccess || dalloc(&pl->d_tof_grp2, grp2.size()) != cudaSuccess ||
      dalloc(&pl->d_tof_grp4, grp4.size()) != cudaSuccess || dalloc(&pl->d_tof_work, 1) != cudaSuccess)
    return PET_ERR_NOMEM;
  if (cudaMemcpy(pl->d_tofw_tab, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(pl->d_tof_grp2, grp2.data(), grp2.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(pl->d_tof_grp4, grp4.data(), grp4.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return PET_ERR_CUDA;
  dp.tofw_tab = pl->d_tofw_tab;
  dp.tof_grp2 = pl->d_tof_grp2;
  dp.tof_ngrp2 = (int)(grp2.size() / 2);
  dp.tof_grp4 = pl->d_tof_grp4;
  dp.tof_ngrp4 = (int)(grp4.size() / 4);
  dp.tof_work = pl->d_tof_work;
  const size_t np = (size_t)(g.nz + 2 * kTofPad) * (g.ny * (size_t)(g.nx + 2 * kTofPad));
  const size_t ntp = (size_t)(g.nz + 2 * kTofPad) * (g.nx * (size_t)(g.ny + 2 * kTofPad));
  if (dalloc(&pl->d_tof_xp, np) != cudaSuccess || dalloc(&pl->d_tof_xtp, ntp) != cudaSuccess ||
      dalloc(&pl->d_tof_gp, np) != cudaSuccess || dalloc(&pl->d_tof_gtp, ntp) != cudaSuccess)
    return PET_ERR_NOMEM;
  if (cudaMemset(pl->d_tof_xp, 0, np * sizeof(float)) != cudaSuccess ||
      cudaMemset(pl->d_tof_xtp, 0, ntp * sizeof(float)) != cudaSuccess ||
      cudaMemset(pl->d_tof_gp, 0, np * sizeof(float)) != cudaSuccess ||
      cudaMemset(pl->d_tof_gtp, 0, ntp * sizeof(float)) != cudaSuccess)
    return PET_ERR_CUDA;
  dp.tof_xp = pl->d_tof_xp;
  dp.tof_xtp = pl->d_tof_xtp;
  dp.tof_gp = pl->d_tof_gp;
  dp.tof_gtp = pl->d_tof_gtp;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pl->device) != cudaSuccess || nsm < 1)
    return PET_ERR_CUDA;
  dp.nsm = nsm;
  return tofk_init_device() == cudaSuccess ? PET_OK : PET_ERR_CUDA;
}

extern "C" pet_status pet_plan_create(const pet_geometry *geom, pet_plan **out) {
  if (!geom || !out) return PET_ERR_ARG;
  *out = nullptr;
  const pet_geometry &g = *geom;
  if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.nrad < 1 || g.nview < 1 || g.nplane < 1) return PET_ERR_ARG;
  if (!(g.dx > 0 && g.dy > 0 && g.dz > 0 && g.drad > 0 && g.rdet > 0)) return PET_ERR_ARG;
  if (!g.z1 || !g.z2) return PET_ERR_ARG;
  if (g.nsubsets < 1 || g.nsubsets > g.nview) return PET_ERR_ARG;
  if (g.ntof > 32) return PET_ERR_UNSUPPORTED;
  if (g.ntof > 1 && !(g.tof_sigma > 0 && g.tof_bin > 0)) return PET_ERR_ARG;
  if (!(g.res_fwhm >= 0.0) || !std::isfinite(g.res_fwhm)) return PET_ERR_ARG;
  GaussTaps taps[3] = {};
  const bool res = g.res_fwhm > 0.0;
  if (res && (!gauss_taps(g.res_fwhm, g.dx, taps[0]) || !gauss_taps(g.res_fwhm, g.dy, taps[1]) ||
              (g.nz > 1 && !gauss_taps(g.res_fwhm, g.dz, taps[2]))))
    return PET_ERR_UNSUPPORTED;
  const long long nvox = (long long)g.nx * g.ny * g.nz;
  const long long nlor = (long long)g.nview * g.nplane * g.nrad;
  if (nvox >= (1LL << 31) || nlor >= (1LL << 31)) return PET_ERR_UNSUPPORTED;
  const double smax = 0.5 * (g.nrad - 1) * g.drad;
  if (!(smax < g.rdet)) return PET_ERR_SHAPE;

  const int V = g.nview, R = g.nrad, P = g.nplane;
  std::vector<float4> view(V), vr((size_t)V * R), plane(P);
  std::vector<float2> aff(V);
  double maxdz = 0.0;
  for (int p = 0; p < P; ++p) maxdz = std::max(maxdz, fabs(g.z2[p] - g.z1[p]));
  for (int v = 0; v < V; ++v) {
    const double phi = v * M_PI / V, c = cos(phi), s = sin(phi);
    const int xd = view_xdrive(g, v);
    const double ua = xd ? -s : c, ub = xd ? c : -s;
    const double da = xd ? g.dx : g.dy, db = xd ? g.dy : g.dx;
    const int Na = xd ? g.nx : g.ny, Nb = xd ? g.ny : g.nx;
    const double a0 = -0.5 * (Na - 1) * da;
    view[v] = make_float4((float)xd, (float)(da * (ub / ua) / db), (float)(da / ua), 0.f);
    double fb_r0 = 0, fb_r1 = 0;
    for (int r = 0; r < R; ++r) {
      const double sr = (r - 0.5 * (R - 1)) * g.drad;
      const double h = sqrt(g.rdet * g.rdet - sr * sr);
      // the axial axis must never drive: |dz|/dz_vox <= 2h|u_a|/delta_a
      if (maxdz / g.dz > 2.0 * h * fabs(ua) / da) return PET_ERR_SHAPE;
      const double Ma = xd ? sr * c : sr * s, Mb = xd ? sr * s : sr * c;
      const double fb0 = (Mb + (a0 - Ma) * (ub / ua)) / db + 0.5 * (Nb - 1);
      const double t0b = (a0 - Ma) / ua;
      vr[(size_t)v * R + r] = make_float4((float)fb0, (float)t0b, (float)(1.0 / (2.0 * h)), 0.f);
      if (r == 0) fb_r0 = fb0;
      if (r == 1) fb_r1 = fb0;
    }
    const double slope = R > 1 ? fb_r1 - fb_r0 : 1.0;
    aff[v] = make_float2((float)fb_r0, (float)(slope != 0.0 ? slope : 1.0));
  }
  for (int p = 0; p < P; ++p) {
    const double zs = (g.z1[p] + g.z2[p]) / (2.0 * g.dz) + 0.5 * (g.nz - 1);
    const double zd = (g.z2[p] - g.z1[p]) / g.dz;
    plane[p] = make_float4((float)zs, (float)zd, (float)(g.z2[p] - g.z1[p]), 0.f);
  }

  pet_plan *pl = new pet_plan();
  pl->g = g;
  pl->z1.assign(g.z1, g.z1 + P);
  pl->z2.assign(g.z2, g.z2 + P);
  pl->g.z1 = pl->z1.data();
  pl->g.z2 = pl->z2.data();
  pl->N = (size_t)nvox;
  pl->T = g.ntof > 1 ? g.ntof : 1;
  cudaGetDevice(&pl->device);
  pl->vs_max = (V + g.nsubsets - 1) / g.nsubsets;

  DevPlan &dp = pl->dp;
  memset(&dp, 0, sizeof(dp));
  dp.nx = g.nx; dp.ny = g.ny; dp.nz = g.nz;
  dp.nrad = R; dp.nview = V; dp.nplane = P; dp.T = pl->T; dp.nsub = g.nsubsets;
  if (pl->T > 1) {
    const double amax = 3.0 / sqrt(2.0);
    dp.tof_inv = (float)(1.0 / (sqrt(2.0) * g.tof_sigma));
    dp.tof_e0 = (float)(-0.5 * pl->T * g.tof_bin);
    dp.tof_w = (float)g.tof_bin;
    dp.tof_amax = (float)amax;
    dp.tof_erfc_amax = (float)erfc(amax);
    dp.tof_half_norm = (float)(1.0 / (2.0 * erf(amax)));
    dp.erfc_scale = (float)(kErfcTab / amax);
  }
  // any fused-gradient launch (up to 16 parts per LOR) has at most this many blocks
  const int gb_all = (int)((16 * nlor + kBlock - 1) / kBlock) + 1;
  const int rb = ratio_blocks(dp, -1);
  pl->npart = std::max({gb_all, rb, rdp_blocks(g.nx, g.ny, g.nz, 2), 4 * nrmse_blocks(pl->N), 1});
  bool ok = dalloc(&pl->d_view, V) == cudaSuccess && dalloc(&pl->d_vr, (size_t)V * R) == cudaSuccess &&
            dalloc(&pl->d_plane, P) == cudaSuccess && dalloc(&pl->d_aff, V) == cudaSuccess &&
            dalloc(&pl->d_m, (size_t)nlor) == cudaSuccess && dalloc(&pl->d_sens, pl->N) == cudaSuccess &&
            dalloc(&pl->d_sens_sub, pl->N * g.nsubsets) == cudaSuccess &&
            dalloc(&pl->d_xT, pl->N) == cudaSuccess && dalloc(&pl->d_gT, pl->N) == cudaSuccess &&
            dalloc(&pl->d_img, pl->N) == cudaSuccess &&
            dalloc(&pl->d_part, (size_t)pl->npart) == cudaSuccess && dalloc(&pl->d_err, 1) == cudaSuccess &&
            dalloc(&pl->d_fpart, (size_t)max_blocks(pl->N)) == cudaSuccess &&
            dalloc(&pl->d_fscalar, 4) == cudaSuccess;
  pl->res = res;
  for (int a = 0; a < 3; ++a) pl->taps[a] = taps[a];
  if (ok && res) ok = dalloc(&pl->d_xs, pl->N) == cudaSuccess && dalloc(&pl->d_rtmp, pl->N) == cudaSuccess;
  if (!ok) { plan_free(pl); return PET_ERR_NOMEM; }
  if (cudaMemcpy(pl->d_view, view.data(), V * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(pl->d_vr, vr.data(), vr.size() * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(pl->d_plane, plane.data(), P * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(pl->d_aff, aff.data(), V * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(pl->d_err, 0, sizeof(int)) != cudaSuccess) {
    plan_free(pl);
    return PET_ERR_CUDA;
  }
  dp.view = pl->d_view; dp.vr = pl->d_vr; dp.plane = pl->d_plane;
  dp.m = pl->d_m; dp.err = pl->d_err;
  pl->dd.view_aff = pl->d_aff;
  if (pl->T > 1) {
    const double amax = 3.0 / sqrt(2.0);
    std::vector<float> tab(kErfcTab + 1);
    for (int j = 0; j <= kErfcTab; ++j) tab[j] = (float)erfc(amax * j / kErfcTab);
    if (dalloc(&pl->d_erfc_tab, kErfcTab + 1) != cudaSuccess) { plan_free(pl); return PET_ERR_NOMEM; }
    if (cudaMemcpy(pl->d_erfc_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      plan_free(pl);
      return PET_ERR_CUDA;
    }
    dp.erfc_tab = pl->d_erfc_tab;
    dp.tof_erfc_amax = tab[kErfcTab];
  }
  if (pl->T > 1 && pl->T <= kTofMaxBins) {
    pet_status e = build_tof_window(pl, plane);
    if (e != PET_OK) { plan_free(pl); return e; }
  }
  {
    // plane groups by axial slope, sorted by axial centre (deterministic backprojector)
    std::vector<int> order(P);
    for (int p = 0; p < P; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      if (plane[a].y != plane[b].y) return plane[a].y < plane[b].y;
      return plane[a].x < plane[b].x;
    });
    std::vector<int2> groups;
    std::vector<float> gzd, gzs(P);
    for (int k = 0; k < P; ++k) {
      gzs[k] = plane[order[k]].x;
      if (k == 0 || plane[order[k]].y != plane[order[k - 1]].y) {
        groups.push_back(make_int2(k, 0));
        gzd.push_back(plane[order[k]].y);
      }
      groups.back().y += 1;
    }
    const int ng = (int)groups.size();
    if (dalloc(&pl->d_groups, ng) != cudaSuccess || dalloc(&pl->d_gzd, ng) != cudaSuccess ||
        dalloc(&pl->d_gplane, P) != cudaSuccess || dalloc(&pl->d_gzs, P) != cudaSuccess) {
      plan_free(pl);
      return PET_ERR_NOMEM;
    }
    if (cudaMemcpy(pl->d_groups, groups.data(), ng * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(pl->d_gzd, gzd.data(), ng * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(pl->d_gplane, order.data(), P * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(pl->d_gzs, gzs.data(), P * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      plan_free(pl);
      return PET_ERR_CUDA;
    }
    pl->dd.ngroups = ng;
    pl->dd.groups = pl->d_groups;
    pl->dd.gzd = pl->d_gzd;
    pl->dd.gplane = pl->d_gplane;
    pl->dd.gzs = pl->d_gzs;
  }
  *out = pl;
  return PET_OK;
}

extern "C" void pet_plan_destroy(pet_plan *plan) { plan_free(plan); }

extern "C" const float *pet_plan_mult(const pet_plan *plan) { return plan ? plan->d_m : nullptr; }

extern "C" const float *pet_plan_sensitivity(const pet_plan *plan, int subset) {
  if (!plan || subset < -1 || subset >= plan->g.nsubsets) return nullptr;
  return subset < 0 ? plan->d_sens : plan->d_sens_sub + plan->N * (size_t)subset;
}

extern "C" pet_status pet_subset_size(const pet_plan *plan, int subset, int *nviews) {
  if (!plan || !nviews || subset < -1 || subset >= plan->g.nsubsets) return PET_ERR_ARG;
  *nviews = subset < 0 ? plan->g.nview
                       : (plan->g.nview - subset + plan->g.nsubsets - 1) / plan->g.nsubsets;
  return PET_OK;
}

namespace petgb {
// x (canonical) -> plan scratch xT (x fastest becomes y fastest)
cudaError_t to_frames(pet_plan *p, const float *x, cudaStream_t st) {
  return launch_transpose(x, p->d_xT, p->g.nx, p->g.ny, p->g.nz, 0, 0, st);
}
// g += transpose(gT), leaving gT zeroed
cudaError_t from_frames(pet_plan *p, float *g, cudaStream_t st) {
  return launch_transpose(p->d_gT, g, p->g.nx, p->g.ny, p->g.nz, 1, 2, st);
}
cudaError_t zero_accumulators(pet_plan *p, float *g, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(g, 0, p->N * sizeof(float), st);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(p->d_gT, 0, p->N * sizeof(float), st);
}
cudaError_t prepare_image(pet_plan *p, const float *x, const float **img, cudaStream_t st) {
  *img = x;
  if (p->res) {
    cudaError_t e = launch_gauss(p->taps, p->g.nx, p->g.ny, p->g.nz, x, p->d_xs, p->d_rtmp, st);
    if (e != cudaSuccess) return e;
    *img = p->d_xs;
  }
  return to_frames(p, *img, st);
}
cudaError_t apply_res(pet_plan *p, float *g, cudaStream_t st) {
  if (!p->res) return cudaSuccess;
  return launch_gauss(p->taps, p->g.nx, p->g.ny, p->g.nz, g, g, p->d_rtmp, st);
}
}  // namespace petgb

extern "C" pet_status pet_plan_set_data(pet_plan *plan, const void *y, pet_ytype yt, const float *r,
                                        const float *mu, const float *sens_lor, void *stream) {
  if (!plan || !y || !r || (int)yt < 0 || (int)yt > 2) return PET_ERR_ARG;
  cudaStream_t st = S(stream);
  DevPlan &dp = plan->dp;
  dp.y = y;
  dp.yt = (int)yt;
  dp.r = r;
  if (mu) PET_CK(launch_transpose(mu, plan->d_xT, plan->g.nx, plan->g.ny, plan->g.nz, 0, 0, st));
  PET_CK(launch_mult(dp, mu, plan->d_xT, sens_lor, plan->d_m, st));
  // sensitivity images with the deterministic backprojector (ones)
  PET_CK(launch_back_det(dp, plan->dd, -1, nullptr, plan->d_sens, 1, st));
  PET_CK(apply_res(plan, plan->d_sens, st));
  for (int s = 0; s < plan->g.nsubsets; ++s) {
    PET_CK(launch_back_det(dp, plan->dd, s, nullptr, plan->d_sens_sub + plan->N * (size_t)s, 1, st));
    PET_CK(apply_res(plan, plan->d_sens_sub + plan->N * (size_t)s, st));
  }
  PET_CK(cudaStreamSynchronize(st));
  plan->has_data = true;
  return PET_OK;
}

extern "C" pet_status pet_plan_set_counts(pet_plan *plan, const void *y, pet_ytype yt, const float *r) {
  if (!plan || !y || !r || (int)yt < 0 || (int)yt > 2) return PET_ERR_ARG;
  if (!plan->has_data) return PET_ERR_STATE;
  plan->dp.y = y;
  plan->dp.yt = (int)yt;
  plan->dp.r = r;
  return PET_OK;
}

extern "C" pet_status pet_plan_check(pet_plan *plan, void *stream) {
  if (!plan) return PET_ERR_ARG;
  int h = 0;
  PET_CK(cudaStreamSynchronize(S(stream)));
  PET_CK(cudaMemcpy(&h, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  PET_CK(cudaMemset(plan->d_err, 0, sizeof(int)));
  return h ? PET_ERR_INFEASIBLE : PET_OK;
}

static bool bad_subset(const pet_plan *p, int s) { return s < -1 || s >= p->g.nsubsets; }

extern "C" pet_status pet_forward(pet_plan *plan, int subset, const float *x, float *out, void *stream) {
  if (!plan || !x || !out || bad_subset(plan, subset)) return PET_ERR_ARG;
  if (!plan->has_data) return PET_ERR_STATE;
  cudaStream_t st = S(stream);
  const float *img = nullptr;
  PET_CK(prepare_image(plan, x, &img, st));
  PET_CK(launch_forward(plan->dp, subset, img, plan->d_xT, out, st));
  return PET_OK;
}

extern "C" pet_status pet_back(pet_plan *plan, int subset, const float *q, float *g, int deterministic,
                               void *stream) {
  if (!plan || !q || !g || bad_subset(plan, subset)) return PET_ERR_ARG;
  if (!plan->has_data) return PET_ERR_STATE;
  cudaStream_t st = S(stream);
  if (deterministic) {
    PET_CK(launch_back_det(plan->dp, plan->dd, subset, q, g, 0, st));
    PET_CK(apply_res(plan, g, st));
    return PET_OK;
  }
  PET_CK(zero_accumulators(plan, g, st));
  PET_CK(launch_back(plan->dp, subset, q, g, plan->d_gT, st));
  PET_CK(from_frames(plan, g, st));
  PET_CK(apply_res(plan, g, st));
  return PET_OK;
}

// Compact-sinogram temporary for the deterministic objective path, grown on demand.
static pet_status ensure_qtmp(pet_plan *p, int subset) {
  const int nv = subset < 0 ? p->g.nview : p->vs_max;
  const size_t n = (size_t)nv * p->g.nplane * p->g.nrad * p->T;
  if (p->qtmp_cap >= n) return PET_OK;
  cudaFree(p->d_qtmp);
  p->d_qtmp = nullptr;
  p->qtmp_cap = 0;
  if (dalloc(&p->d_qtmp, n) != cudaSuccess) return PET_ERR_NOMEM;
  p->qtmp_cap = n;
  return PET_OK;
}

extern "C" pet_status pet_objective_grad(pet_plan *plan, int subset, const float *x, float *g, double *obj,
                                         const pet_rdp_params *prior, int flags, void *stream) {
  if (!plan || !x || bad_subset(plan, subset)) return PET_ERR_ARG;
  const bool obj_only = (flags & PET_OBJ_ONLY) != 0;
  if (!obj_only && !g) return PET_ERR_ARG;
  if (!plan->has_data) return PET_ERR_STATE;
  if (prior && (prior->nx != plan->g.nx || prior->ny != plan->g.ny || prior->nz != plan->g.nz))
    return PET_ERR_ARG;
  cudaStream_t st = S(stream);
  const float *img = nullptr;
  PET_CK(prepare_image(plan, x, &img, st));
  int nparts = 0;
  if (flags & PET_GRAD_DETERMINISTIC && !obj_only) {
    pet_status e = ensure_qtmp(plan, subset);
    if (e != PET_OK) return e;
    float *ax = plan->d_qtmp;
    PET_CK(launch_forward(plan->dp, subset, img, plan->d_xT, ax, st));
    nparts = ratio_blocks(plan->dp, subset);
    PET_CK(launch_ratio(plan->dp, subset, ax, ax, obj ? plan->d_part : nullptr, MODE_GRAD, st));
    PET_CK(launch_back_det(plan->dp, plan->dd, subset, ax, g, 0, st));
    PET_CK(apply_res(plan, g, st));
  } else {
    if (!obj_only) PET_CK(zero_accumulators(plan, g, st));
    PET_CK(launch_grad(plan->dp, subset, nullptr, img, plan->d_xT, g, plan->d_gT, obj ? plan->d_part : nullptr,
                       obj_only ? MODE_OBJ : MODE_GRAD, &nparts, st));
    if (!obj_only) {
      PET_CK(from_frames(plan, g, st));
      PET_CK(apply_res(plan, g, st));
    }
  }
  if (obj) PET_CK(launch_reduce_sum(plan->d_part, nparts, obj, 0, st));
  if (prior) {
    RdpArgs a = make_rdp_args(*prior);
    a.zch = plan->rdp_zch;
    int nb = 0;
    PET_CK(launch_rdp(a, x, obj_only ? nullptr : g, nullptr, obj ? plan->d_part : nullptr, 1, &nb, st));
    if (obj) PET_CK(launch_reduce_sum(plan->d_part, nb, obj, 1, st));
  }
  return PET_OK;
}

extern "C" pet_status pet_em_update(pet_plan *plan, int subset, float *x, void *stream) {
  if (!plan || !x || subset < 0 || subset >= plan->g.nsubsets) return PET_ERR_ARG;
  if (!plan->has_data) return PET_ERR_STATE;
  cudaStream_t st = S(stream);
  float *bp = plan->d_img;
  const float *img = nullptr;
  PET_CK(prepare_image(plan, x, &img, st));
  PET_CK(zero_accumulators(plan, bp, st));
  PET_CK(launch_grad(plan->dp, subset, nullptr, img, plan->d_xT, bp, plan->d_gT, nullptr, MODE_EM, nullptr, st));
  PET_CK(from_frames(plan, bp, st));
  PET_CK(apply_res(plan, bp, st));
  PET_CK(launch_em_apply(x, bp, plan->d_sens_sub + plan->N * (size_t)subset, plan->N, st));
  return PET_OK;
}

extern "C" pet_status pet_rdp(const pet_rdp_params *p, const float *x, float *grad, float *hdiag,
                              double *val, int accumulate, void *stream) {
  if (!p || !x || p->nx < 1 || p->ny < 1 || p->nz < 1) return PET_ERR_ARG;
  cudaStream_t st = S(stream);
  RdpArgs a = make_rdp_args(*p);
  double *part = nullptr;
  const int nb = rdp_blocks(p->nx, p->ny, p->nz);
  if (val && cudaMallocAsync((void **)&part, nb * sizeof(double), st) != cudaSuccess) return PET_ERR_NOMEM;
  cudaError_t e = launch_rdp(a, x, grad, hdiag, part, accumulate & PET_RDP_ACC_GRAD, nullptr, st);
  if (e == cudaSuccess && val) e = launch_reduce_sum(part, nb, val, (accumulate & PET_RDP_ACC_VAL) ? 1 : 0, st);
  if (part) cudaFreeAsync(part, st);
  return e == cudaSuccess ? PET_OK : PET_ERR_CUDA;
}

extern "C" pet_status pet_precond(pet_plan *plan, const float *x, const float *hdiag_betaS, float alpha,
                                  float delta_rel, float *D, void *stream) {
  if (!plan || !x || !D) return PET_ERR_ARG;
  if (!plan->has_data) return PET_ERR_STATE;
  cudaStream_t st = S(stream);
  PET_CK(launch_max(x, plan->N, plan->d_fpart, plan->d_fscalar, st));
  PET_CK(launch_precond(x, plan->d_sens, hdiag_betaS, alpha, plan->d_fscalar, delta_rel, D, plan->N, st));
  return PET_OK;
}

extern "C" pet_status pet_nrmse(const float *x, const float *ref, const uint8_t *mask, const uint8_t *bg,
                                size_t n, double *out, void *stream) {
  if (!x || !ref || !mask || !bg || !out || n == 0) return PET_ERR_ARG;
  cudaStream_t st = S(stream);
  double *part = nullptr;
  const int nb = nrmse_blocks(n);
  if (cudaMallocAsync((void **)&part, 4 * nb * sizeof(double), st) != cudaSuccess) return PET_ERR_NOMEM;
  cudaError_t e = launch_nrmse(x, ref, mask, bg, n, part, out, st);
  cudaFreeAsync(part, st);
  return e == cudaSuccess ? PET_OK : PET_ERR_CUDA;
}

extern "C" pet_status pet_plan_set_grad_shape(pet_plan *plan, int planes_per_thread, int parts) {
  if (!plan) return PET_ERR_ARG;
  const bool kok = planes_per_thread == 0 || planes_per_thread == 1 ||
                   ((planes_per_thread == 2 || planes_per_thread == 4) && planes_per_thread <= max_planes(plan->dp));
  const bool sok = parts == 0 || ((parts == 1 || parts == 2 || parts == 4 || parts == 8 || parts == 16) &&
                                   parts <= max_split(plan->dp));
  if (!kok || !sok) return PET_ERR_ARG;
  plan->dp.grad_k = planes_per_thread;
  plan->dp.grad_split = parts;
  return PET_OK;
}

extern "C" pet_status pet_plan_set_rdp_tile(pet_plan *plan, int slices) {
  if (!plan || !(slices == 0 || slices == 2 || slices == 4 || slices == 8)) return PET_ERR_ARG;
  plan->rdp_zch = slices ? slices : kRdpZchDefault;
  return PET_OK;
}

extern "C" pet_status pet_plan_autotune(pet_plan *plan, void *stream, int *planes_per_thread, int *parts) {
  if (!plan) return PET_ERR_ARG;
  if (!plan->has_data) return PET_ERR_STATE;
  cudaStream_t st = S(stream);
  const int ks[3] = {1, 2, 4}, ss[5] = {1, 2, 4, 8, 16};
  float *x = plan->d_img, *g = nullptr;
  if (dalloc(&g, plan->N) != cudaSuccess) return PET_ERR_NOMEM;  // setup-time temporary
  if (launch_fill(x, plan->N, 1.f, st) != cudaSuccess) { cudaFree(g); return PET_ERR_CUDA; }
  cudaEvent_t e0, e1;
  if (to_frames(plan, x, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess) {
    cudaFree(g);
    return PET_ERR_CUDA;
  }
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaFree(g);
    return PET_ERR_CUDA;
  }
  const int old_k = plan->dp.grad_k, old_s = plan->dp.grad_split;
  // Three rounds over every valid shape, 12 timed launches each (on four subsets in turn)
  // after 2 untimed ones; a shape's time is its fastest round (the best shapes differ by a
  // few percent).
  float tmin[3][5];
  for (auto &row : tmin)
    for (float &t : row) t = 1e30f;
  for (int round = 0; round < 3; ++round)
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 5; ++b) {
      if (ks[a] > max_planes(plan->dp) || ss[b] > max_split(plan->dp)) continue;
      plan->dp.grad_k = ks[a];
      plan->dp.grad_split = ss[b];
      float ms = 0.f;
      bool fail = false;
      for (int it = 0; it < 14 && !fail; ++it) {
        if (it == 2) fail |= cudaEventRecord(e0, st) != cudaSuccess;
        // four subsets spread over the views (their view angles, hence driving axes and
        // TOF directions, differ)
        const int sub = ((it % 4) * plan->g.nsubsets) / 4;
        fail |= launch_grad(plan->dp, sub, nullptr, x, plan->d_xT, g, plan->d_gT, nullptr, MODE_GRAD, nullptr, st) !=
                cudaSuccess;
      }
      fail |= cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess;
      if (fail) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamSynchronize(st);
        cudaFree(g);
        plan->dp.grad_k = old_k;
        plan->dp.grad_split = old_s;
        return PET_ERR_CUDA;
      }
      tmin[a][b] = std::min(tmin[a][b], ms);
    }
  float best = 1e30f;
  int bk = 1, bs = 1;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 5; ++b)
      if (tmin[a][b] < best) { best = tmin[a][b]; bk = ks[a]; bs = ss[b]; }
  // RDP stencil tile: slices per block, timed on the same image (gradient only)
  pet_rdp_params rp = {};
  rp.nx = plan->g.nx; rp.ny = plan->g.ny; rp.nz = plan->g.nz;
  rp.dx = plan->g.dx; rp.dy = plan->g.dy; rp.dz = plan->g.dz;
  rp.gamma = 2.f; rp.eps = 1e-3f; rp.scale = 1.f; rp.kappa = nullptr;
  RdpArgs ra = make_rdp_args(rp);
  const int zs[3] = {2, 4, 8};
  float zbest = 1e30f;
  int bz = kRdpZchDefault;
  for (int round = 0; round < 2; ++round)
    for (int zch : zs) {
      ra.zch = zch;
      float ms = 0.f;
      bool fail = false;
      for (int it = 0; it < 12 && !fail; ++it) {
        if (it == 2) fail |= cudaEventRecord(e0, st) != cudaSuccess;
        fail |= launch_rdp(ra, x, g, nullptr, nullptr, 0, nullptr, st) != cudaSuccess;
      }
      fail |= cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess;
      if (fail) break;
      if (ms < zbest) { zbest = ms; bz = zch; }
    }
  plan->rdp_zch = bz;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(g);
  plan->dp.grad_k = bk;
  plan->dp.grad_split = bs;
  PET_CK(zero_accumulators(plan, plan->d_img, st));  // leave the transposed accumulator clear
  PET_CK(cudaStreamSynchronize(st));
  if (planes_per_thread) *planes_per_thread = bk;
  if (parts) *parts = bs;
  return PET_OK;
}

extern "C" pet_status pet_ratio(pet_plan *plan, int subset, const float *ax, float *q, double *obj, int em,
                                void *stream) {
  if (!plan || !ax || bad_subset(plan, subset) || (!q && !obj)) return PET_ERR_ARG;
  if (!plan->has_data) return PET_ERR_STATE;
  cudaStream_t st = S(stream);
  const int nparts = ratio_blocks(plan->dp, subset);
  PET_CK(launch_ratio(plan->dp, subset, ax, q, obj ? plan->d_part : nullptr, em ? MODE_EM : MODE_GRAD, st));
  if (obj) PET_CK(launch_reduce_sum(plan->d_part, nparts, obj, 0, st));
  return PET_OK;
}
