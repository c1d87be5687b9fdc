// Host-side plan object behind the opaque pet_plan handle.
#pragma once

#include <vector>

#include "pet_internal.cuh"

struct pet_plan {
  pet_geometry g;             // copy; z1/z2 point into the vectors below
  std::vector<double> z1, z2;
  size_t N = 0;               // voxels
  int T = 1;                  // TOF bins (1: non-TOF)
  int vs_max = 0;             // views in the largest subset
  int device = 0;
  int rdp_zch = petgb::kRdpZchDefault;  // slices per RDP stencil block (autotuned)
  bool has_data = false;
  petgb::DevPlan dp;
  petgb::DevPlanDet dd;
  // geometry tables
  float4 *d_view = nullptr, *d_vr = nullptr, *d_plane = nullptr;
  float2 *d_aff = nullptr;
  int2 *d_groups = nullptr;    // deterministic backprojector: plane groups
  float *d_gzd = nullptr, *d_gzs = nullptr;
  int *d_gplane = nullptr;
  float *d_erfc_tab = nullptr;  // TOF: erfc table
  float4 *d_tofw_tab = nullptr; // TOF: rows of the interpolated bin-weight table (windowed kernel)
  int *d_tof_grp2 = nullptr;    // TOF: plane pairs of equal axial slope
  int *d_tof_grp4 = nullptr;    // TOF: plane quadruples of equal axial slope
  unsigned long long *d_tof_work = nullptr;  // TOF: work counter of the persistent kernel
  float *d_tof_xp = nullptr, *d_tof_xtp = nullptr;  // TOF: zero-padded image frames
  float *d_tof_gp = nullptr, *d_tof_gtp = nullptr;  // TOF: zero-padded gradient accumulators
  // derived data
  float *d_m = nullptr;         // [V][P][R] multiplicative factors
  float *d_sens = nullptr;      // [N] A^T 1
  float *d_sens_sub = nullptr;  // [n][N] A_s^T 1
  // scratch: driving-frame image and gradient (x-driven views), image temp, partials
  float *d_xT = nullptr, *d_gT = nullptr, *d_img = nullptr;
  double *d_part = nullptr;
  int npart = 0;
  int *d_err = nullptr;
  float *d_fpart = nullptr, *d_fscalar = nullptr;
  float *d_qtmp = nullptr;
  size_t qtmp_cap = 0;
  // image-space resolution model (geometry res_fwhm > 0): taps per axis, G x and a temp
  bool res = false;
  petgb::GaussTaps taps[3];
  float *d_xs = nullptr, *d_rtmp = nullptr;
};

namespace petgb {
cudaError_t to_frames(pet_plan *p, const float *x, cudaStream_t st);
cudaError_t from_frames(pet_plan *p, float *g, cudaStream_t st);
cudaError_t zero_accumulators(pet_plan *p, float *g, cudaStream_t st);
// The image the projector reads: x itself, or G x in plan scratch with the resolution
// model; either way the transposed copy in d_xT is refreshed.
cudaError_t prepare_image(pet_plan *p, const float *x, const float **img, cudaStream_t st);
// g <- G g when the plan has a resolution model (after the accumulators are combined).
cudaError_t apply_res(pet_plan *p, float *g, cudaStream_t st);
}  // namespace petgb
