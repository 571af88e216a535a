// Host side of the 2D stencil: validation helpers, functor mapping (Sec. 4.2, Sec. 5.2),
// choice of the specialised kernel and tile shape, and dispatch by storage type.
#include <cmath>
#include <cstdio>
#include <cstring>

#include <atomic>
#include <cudaTypedefs.h>

#include "cs_stencil2d_kernels.cuh"

namespace cs {

int stencil2d_launch_f32(const Stencil2DConfig* cfg, const void* in, void* out, cudaStream_t s);
int stencil2d_launch_f64(const Stencil2DConfig* cfg, const void* in, void* out, cudaStream_t s);
int stencil2d_group_f32(const Stencil2DConfig* const* cfgs, const void* const* ins, void* const* outs,
                        int count, cudaStream_t s);
int stencil2d_group_f64(const Stencil2DConfig* const* cfgs, const void* const* ins, void* const* outs,
                        int count, cudaStream_t s);

namespace {

// Effective weights of the compiled-in user functions, in the Sec. 5.2 ordering.
int map_function(Stencil2DConfig* cfg) {
  const double c = cfg->coe[0];
  switch (cfg->fn) {
    case CS_FN_CENTRAL_D2X: {  // Sec. 4.2: second-order central difference in x
      const double w[3] = {c, -2.0 * c, c};
      memcpy(cfg->weights, w, sizeof w);
      cfg->variant = 4;
      return CS_OK;
    }
    case CS_FN_CH_NONLIN_LAP: {  // Laplacian of u^3 - u (staged transform)
      const double w[9] = {0, c, 0, c, -4.0 * c, c, 0, c, 0};
      memcpy(cfg->weights, w, sizeof w);
      cfg->variant = 12;
      return CS_OK;
    }
    case CS_FN_CUBIC_MINUS_LAP: {  // u^3 - u - Laplacian(u)
      const double w[9] = {0, -c, 0, -c, 4.0 * c, -c, 0, -c, 0};
      memcpy(cfg->weights, w, sizeof w);
      cfg->variant = 13;
      return CS_OK;
    }
    default:
      return set_error(CS_EINVAL, "unknown user function %d", cfg->fn);
  }
}

}  // namespace

int stencil2d_prepare(Stencil2DConfig* cfg) {
  cfg->d_weights = nullptr;
  cfg->d_weights_f = nullptr;
  cfg->d_status = nullptr;
  cfg->aux = nullptr;
  cfg->ev_fork = cfg->ev_join = nullptr;
  cfg->status_seen = 0;
  cfg->stall_from = -1;
  cfg->variant = -1;
  cfg->tmap_in = nullptr;
  if (cfg->tile_rows != 32 && cfg->tile_rows != 64) cfg->tile_rows = 64;
  cfg->use_tma = 1;
  const int W = cfg->left + cfg->right + 1, H = cfg->top + cfg->bottom + 1;
  if (cfg->fn != CS_FN_NONE) {
    int rc = map_function(cfg);
    if (rc != CS_OK) return rc;
  } else {
    // smallest specialisation with the same extents whose mask covers every non-zero weight
    uint32_t mask = 0;
    bool fits = W * H <= 32;
    if (fits)
      for (int i = 0; i < W * H; ++i)
        if (cfg->weights[i] != 0.0) mask |= 1u << i;
    int best = -1, best_taps = 1 << 30;
    for (int v = 0; fits && v < s2d::kNumSpecs; ++v) {
      const s2d::SpecDesc& sd = s2d::kSpecs[v];
      if (sd.xform || sd.epi) continue;
      if (sd.L != cfg->left || sd.R != cfg->right || sd.T != cfg->top || sd.B != cfg->bottom) continue;
      if ((mask & ~sd.mask) != 0) continue;
      const int taps = __builtin_popcount(sd.mask);
      if (taps < best_taps) { best = v; best_taps = taps; }
    }
    cfg->variant = best;
  }
  if (cfg->variant < 0) {  // generic kernel: weights in device memory
    const size_t n = static_cast<size_t>(W) * H;
    cudaError_t e = cudaMalloc(&cfg->d_weights, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&cfg->d_weights_f, n * sizeof(float));
    if (e != cudaSuccess) {
      stencil2d_release(cfg);
      return cuda_error(e, "cudaMalloc(weights)");
    }
    float wf[(2 * CS_MAX_EXTENT + 1) * (2 * CS_MAX_EXTENT + 1)];
    for (size_t i = 0; i < n; ++i) wf[i] = static_cast<float>(cfg->weights[i]);
    CS_CUDA_TRY(cudaMemcpy(cfg->d_weights, cfg->weights, n * sizeof(double), cudaMemcpyHostToDevice));
    CS_CUDA_TRY(cudaMemcpy(cfg->d_weights_f, wf, n * sizeof(float), cudaMemcpyHostToDevice));
  }
  // double-float eligibility: every non-zero weight in [2^-60, 2^50), at least one non-zero
  {
    const int nw = (cfg->fn != CS_FN_NONE) ? 9 : W * H;
    bool any = false, fits = true;
    for (int i = 0; i < nw; ++i) {
      const double a = fabs(cfg->weights[i]);
      if (a == 0.0) continue;
      any = true;
      if (!(a >= 0x1p-60 && a < 0x1p50)) fits = false;
    }
    cfg->dd_ok = any && fits;
  }
  // exact digit path: plain weighted specialisations whose weights are c * n_k with integers
  // n_k, sum |n_k| <= 64 (so digit sums stay below 2^24), to 2^-44 of the largest weight
  cfg->ix_ok = 0;
  if (cfg->variant >= 0 && cfg->fn == CS_FN_NONE && !s2d::kSpecs[cfg->variant].xform &&
      !s2d::kSpecs[cfg->variant].epi && cfg->dd_ok) {
    const int nw = W * H;
    double wmin = 0.0, wmax = 0.0;
    for (int i = 0; i < nw; ++i) {
      const double a = fabs(cfg->weights[i]);
      if (a > 0.0 && (wmin == 0.0 || a < wmin)) wmin = a;
      if (a > wmax) wmax = a;
    }
    for (int m = 1; m <= 64 && !cfg->ix_ok; ++m) {
      const double c = wmin / m;
      long long total = 0;
      bool ok = true;
      for (int i = 0; i < nw && ok; ++i) {
        const double r = cfg->weights[i] / c;
        const long long k = llround(r);
        if (fabs(cfg->weights[i] - static_cast<double>(k) * c) > 0x1p-44 * wmax) ok = false;
        total += k < 0 ? -k : k;
        if (total > 64) ok = false;
        cfg->ix_n[i] = static_cast<int>(k);
      }
      if (ok) {
        cfg->ix_ok = 1;
        cfg->ix_c = c;
      }
    }
  }
  // the cubic user function (variant 13): weights c * (0, -1, 0, -1, 4, -1, 0, -1, 0); its cubic
  // term joins the digit sum as an integer in units of c (see ixf_tile_ok), for |c| in [4, 2^40]
  if (cfg->fn == CS_FN_CUBIC_MINUS_LAP && cfg->dd_ok) {
    const double c = cfg->coe[0];
    if (fabs(c) >= 4.0 && fabs(c) <= 0x1p40) {
      const int n[9] = {0, -1, 0, -1, 4, -1, 0, -1, 0};
      for (int i = 0; i < 9; ++i) cfg->ix_n[i] = n[i];
      cfg->ix_c = c;
      cfg->ix_ok = 1;
    }
  }
  // the plan's timeout counter for its TMA sweeps (read by cs_plan_check)
  cudaError_t e = cudaMalloc(&cfg->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(cfg->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    stencil2d_release(cfg);
    return cuda_error(e, "cudaMalloc(status)");
  }
  if (cfg->dtype == CS_F64 && cfg->bc != CS_BC_PERIODIC && cfg->ix_ok) {
    cudaError_t e2 = cudaStreamCreateWithFlags(&cfg->aux, cudaStreamNonBlocking);
    if (e2 == cudaSuccess) e2 = cudaEventCreateWithFlags(&cfg->ev_fork, cudaEventDisableTiming);
    if (e2 == cudaSuccess) e2 = cudaEventCreateWithFlags(&cfg->ev_join, cudaEventDisableTiming);
    if (e2 != cudaSuccess) {
      stencil2d_release(cfg);
      return cuda_error(e2, "border stream");
    }
  }
  int choice;
  if (tune_lookup(stencil2d_shape_key(cfg), &choice)) stencil2d_set_tile_choice(cfg, choice);
  return CS_OK;
}

void stencil2d_release(Stencil2DConfig* cfg) {
  if (cfg->d_weights) cudaFree(cfg->d_weights);
  if (cfg->d_weights_f) cudaFree(cfg->d_weights_f);
  if (cfg->d_status) cudaFree(cfg->d_status);
  if (cfg->ev_fork) cudaEventDestroy(cfg->ev_fork);
  if (cfg->ev_join) cudaEventDestroy(cfg->ev_join);
  if (cfg->aux) cudaStreamDestroy(cfg->aux);
  cfg->d_weights = nullptr;
  cfg->d_weights_f = nullptr;
  cfg->d_status = nullptr;
  cfg->aux = nullptr;
  cfg->ev_fork = cfg->ev_join = nullptr;
}

// Waits for the stream, then reads the plan's timeout counter: a TMA sweep whose bounded
// mbarrier wait ran out since the last check left part of its output unwritten.
int stencil2d_check(const Stencil2DConfig* cfg, cudaStream_t s) {
  CS_CUDA_TRY(cudaStreamSynchronize(s));
  if (!cfg->d_status) return CS_OK;
  int count = 0;
  CS_CUDA_TRY(cudaMemcpy(&count, cfg->d_status, sizeof count, cudaMemcpyDeviceToHost));
  if (count != cfg->status_seen) {
    const int ran_out = count - cfg->status_seen;
    cfg->status_seen = count;
    return set_error(CS_ETIMEOUT, "a TMA sweep's bounded wait ran out in %d CTA(s): part of the output was not written",
                     ran_out);
  }
  return CS_OK;
}

// Tile / pipeline choices the autotuner times: 0 = cp.async tiles of 32 rows, 1 = cp.async
// tiles of 64 rows, 2 = TMA-pipelined persistent sweep (64-row tiles; aligned buffers only).
int stencil2d_num_tile_choices() { return 3; }

int stencil2d_set_tile_choice(Stencil2DConfig* cfg, int choice) {
  cfg->use_tma = choice == 2;
  cfg->tile_rows = choice == 0 ? 32 : 64;
  return CS_OK;
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::atomic<int> g_encode_state{0};
}  // namespace

int s2d::make_tensor_map(const Stencil2DConfig* cfg, const void* in, int elem_bytes, int cols, int rows) {
  if (g_encode_state.load() == 0) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      g_encode_state.store(-1);
    } else {
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
      g_encode_state.store(1);
    }
  }
  if (g_encode_state.load() < 0) return set_error(CS_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cfg->nx), static_cast<cuuint64_t>(cfg->ny)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(cfg->nx) * elem_bytes};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(cols), static_cast<cuuint32_t>(rows)};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(&cfg->tmap, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        2, const_cast<void*>(in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(CS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  cfg->tmap_in = in;
  return CS_OK;
}

std::string stencil2d_shape_key(const Stencil2DConfig* cfg) {
  char buf[160];
  const int64_t cells = cfg->nx * cfg->ny;
  const int size_class = cells <= (1 << 16) ? 0 : cells <= (1 << 22) ? 1 : 2;
  snprintf(buf, sizeof buf, "stencil2d|%s|v%d_e%d.%d.%d.%d_bc%d_s%d|sm%d",
           cfg->dtype == CS_F32 ? "f32" : "f64", cfg->variant, cfg->left, cfg->right, cfg->top,
           cfg->bottom, cfg->bc, size_class, num_sms());
  return buf;
}

int stencil2d_group(const Stencil2DConfig* const* cfgs, const void* const* ins, void* const* outs,
                    int count, cudaStream_t s) {
  return cfgs[0]->dtype == CS_F32 ? stencil2d_group_f32(cfgs, ins, outs, count, s)
                                  : stencil2d_group_f64(cfgs, ins, outs, count, s);
}

int stencil2d_launch(const Stencil2DConfig* cfg, const void* in, void* out, cudaStream_t s) {
  if (cfg->nx == 0 || cfg->ny == 0) return CS_OK;
  // one launch covers the grid: column tiles (>= 64 columns) in grid.x, row tiles (>= 32 rows) in
  // grid.y, whose limit is 65535
  if ((cfg->nx + 63) / 64 > 0x7fffffff || (cfg->ny + 31) / 32 > 65535)
    return set_error(CS_EUNSUPPORTED, "grid %lld x %lld exceeds one launch (ny <= 2097120); a host-resident plan streams taller grids",
                     (long long)cfg->nx, (long long)cfg->ny);
  return cfg->dtype == CS_F32 ? stencil2d_launch_f32(cfg, in, out, s)
                              : stencil2d_launch_f64(cfg, in, out, s);
}

int stencil2d_launch_rows(const Stencil2DConfig* cfg, const void* in, void* out, int64_t row0,
                          int64_t row1, cudaStream_t s) {
  if (row0 % kStencilBandAlign != 0) return set_error(CS_EINVAL, "internal: band start %lld not aligned", (long long)row0);
  s2d::RowWindow& w = s2d::row_window();
  w.row0 = row0;
  w.row1 = row1;
  const int rc = stencil2d_launch(cfg, in, out, s);
  w = s2d::RowWindow{};
  return rc;
}

}  // namespace cs
