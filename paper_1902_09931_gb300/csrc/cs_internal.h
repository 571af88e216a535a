// Internal declarations shared by the translation units of libcusten_gb (not installed).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "custen_gb.h"

namespace cs {

// ---- errors ---------------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);  // records a thread-local message, returns code
int cuda_error(cudaError_t e, const char* what);  // CS_ECUDA with the CUDA message
#define CS_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return ::cs::cuda_error(_e, #expr); \
  } while (0)

void count_launches(int64_t n);  // adds to cs_launch_count()
int num_sms();                   // SM count of the current device (cached per device)

// ---- tuning table (cs_tune.cpp) ----------------------------------------------------------------
// Key: "<kernel>|<dtype>|<shape class>|sm<count>"  ->  small integer choice.
bool tune_lookup(const std::string& key, int* choice);
void tune_store(const std::string& key, int choice);

// ---- 2D stencil (cs_stencil2d.cu) --------------------------------------------------------------
struct Stencil2DConfig {
  int64_t nx, ny;
  int dir, bc, dtype;
  int left, right, top, bottom;
  int fn;
  double weights[(2 * CS_MAX_EXTENT + 1) * (2 * CS_MAX_EXTENT + 1)];
  double coe[8];
  int num_coe;
  // chosen at create time
  int variant;     // index into the specialisation table, or -1 for the generic kernel
  int tile_rows;   // TY
  double* d_weights;  // device copy for the generic kernel (library-owned), FP64
  float* d_weights_f; // FP32 copy
  int dd_ok;          // weights fit the double-float path (FP64 storage)
  int use_tma;        // tile choice 2: TMA-pipelined persistent sweep (aligned buffers)
  mutable CUtensorMap tmap;      // tensor map of the last input pointer (rebuilt on change)
  mutable const void* tmap_in;
  int ix_ok;          // weights are c * small integers: exact digit path (FP64 storage)
  double ix_c;        // common scale c
  int ix_n[32];       // integer ratios n_k
  int fp64_mode;      // CS_FP64_AUTO or CS_FP64_NATIVE
  int* d_status;      // library-owned counter: CTAs of this plan's TMA sweeps whose bounded wait ran out
  mutable int status_seen;  // counter value at the last cs_plan_check
  int stall_from;     // test hook (cs_plan_debug_stall): CTA-local tile from which the TMA sweep
                      // issues no copies, so its wait runs out; -1 = off
  // non-periodic FP64 digit sweeps: the border tiles run on this stream beside the interior
  // tiles' launch (fork and join by the two events); created with the plan
  cudaStream_t aux;
  cudaEvent_t ev_fork, ev_join;
};
int stencil2d_prepare(Stencil2DConfig* cfg);  // picks variant, allocates generic weights
void stencil2d_release(Stencil2DConfig* cfg);
int stencil2d_launch(const Stencil2DConfig* cfg, const void* in, void* out, cudaStream_t s);
// Writes only output rows [row0, row1) (row0 a multiple of kStencilBandAlign, a multiple of every
// tile height; row1 clipped to ny); reads the input rows those outputs need.
constexpr int64_t kStencilBandAlign = 64;
int stencil2d_launch_rows(const Stencil2DConfig* cfg, const void* in, void* out, int64_t row0,
                          int64_t row1, cudaStream_t s);
int stencil2d_num_tile_choices();
int stencil2d_check(const Stencil2DConfig* cfg, cudaStream_t s);  // CS_ETIMEOUT if a wait ran out
int stencil2d_set_tile_choice(Stencil2DConfig* cfg, int choice);
std::string stencil2d_shape_key(const Stencil2DConfig* cfg);
int stencil2d_group(const Stencil2DConfig* const* cfgs, const void* const* ins, void* const* outs,
                    int count, cudaStream_t s);  // same dtype / variant / tile rows, count <= 64
constexpr int kMaxGroupJobs = 64;

// ---- batched 1D (cs_batch1d.cu) -------------------------------------------------------------
struct Batch1DConfig {
  int64_t num_lines, total_len;
  int bc, dtype, left, right;
  double weights[2 * CS_MAX_EXTENT + 1];
  const int64_t* d_offsets;  // caller-owned
  int32_t* d_seg_line;       // library-owned: line containing element s * kSegTable
  int64_t num_table;
  int choice;                // launch shape index
};
int batch1d_prepare(Batch1DConfig* cfg, cudaStream_t s);
void batch1d_release(Batch1DConfig* cfg);
int batch1d_launch(const Batch1DConfig* cfg, const void* in, void* out, cudaStream_t s);
int batch1d_num_choices();
std::string batch1d_shape_key(const Batch1DConfig* cfg);

// ---- periodic XY WENO advection (cs_weno.cu) ---------------------------------------------------
struct WenoConfig {
  int64_t nx, ny;
  int dtype;
  double hx, hy;
};
int weno_launch(const WenoConfig* cfg, const void* c, const void* u, const void* v, void* out, cudaStream_t s);

// ---- Cahn-Hilliard ADI (cs_ch.cu) -------------------------------------------------------------
struct CHPlan;
int ch_create(CHPlan** out, const cs_ch_desc* d, void* prev, void* cur, void* next);
int ch_step(CHPlan* p, int64_t nsteps, double* h_mass, double* h_energy, cudaStream_t s);
int ch_invariants(CHPlan* p, double* mass, double* energy, cudaStream_t s);
int ch_coarsening(CHPlan* p, double* s_out, double* k1_out, cudaStream_t s);
int ch_fields(CHPlan* p, void** prev, void** cur, int64_t* steps);
int ch_config(CHPlan* p, int32_t* chunks, int32_t* chunk_len);
int ch_set_fields(CHPlan* p, void* prev, void* cur, void* next);
int ch_autotune(CHPlan* p, cudaStream_t s);
void ch_destroy(CHPlan* p);
int ch_solver_check(int64_t n, int P, double a, bool noflux, double* residual);
struct CHBand;
int ch_band_create(CHBand** out, const cs_ch_desc* d, int64_t rows);
int ch_band_rhs(CHBand* b, const void* prev, const void* cur, double* rhs, double* sums, cudaStream_t s);
int ch_band_solve(CHBand* b, const double* in, double* out, cudaStream_t s);
int ch_band_update(CHBand* b, const void* prev, const void* cur, const double* v, void* next, cudaStream_t s);
int ch_partition(const cs_ch_desc* d, int32_t* chunks, int32_t* chunk_len);
int ch_band_ycols_local(CHBand* b, int64_t chunk0, const double* in, double* ends, cudaStream_t s);
int ch_band_ycols_correct(CHBand* b, int64_t chunk0, const double* ends_all, double* v, cudaStream_t s);
void ch_band_destroy(CHBand* b);

}  // namespace cs
