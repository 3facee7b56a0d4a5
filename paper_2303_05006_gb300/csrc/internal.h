// internal.h -- library-private declarations shared by the CUDA translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "../../include/tdbem.h"

#define TDBEM_CUDA_TRY(ctx, call)                                                       \
  do {                                                                                  \
    cudaError_t e__ = (call);                                                           \
    if (e__ != cudaSuccess) {                                                           \
      (ctx)->set_error(std::string(#call) + ": " + cudaGetErrorString(e__));            \
      return (e__ == cudaErrorMemoryAllocation) ? TDBEM_ENOMEM : TDBEM_ECUDA;           \
    }                                                                                   \
  } while (0)

namespace tdbem {

constexpr int kMaxWin = 64;   // max lags of one (observation point, source triangle) pair
constexpr int kNq = 7;        // outer quadrature points per test triangle

// Per-triangle geometry in device memory (structure of arrays).
struct TriGeom {
  double* v;       // [nt][3][3] vertex coordinates
  double* nrm;     // [nt][3] unit normal of the winding (outward)
  double* cen;     // [nt][3] centroid
  double* area;    // [nt]
  double* rad;     // [nt] max centroid-vertex distance
  double* lmax;    // [nt] longest side
  int32_t* edge;   // [nt][3] edge on side k (vertex k -> k+1)
  int8_t* sgn;     // [nt][3] +1 if this triangle is the + triangle of that edge
  double* opp;     // [nt][3][3] vertex opposite side k (the o of that edge's RWG on this triangle)
  double* elen;    // [nt][3] length of side k
};

// Physical and discretisation constants passed by value to kernels.
struct Phys {
  double dt, a;                // time step, c*dt
  double c, eta, eps, mu;
  double theta, zeta, s_jump;
  double chi;                  // weight of the time-differentiated MFIE (1: the paper's CFIE)
  double qb[kNq][3], qw[kNq];  // outer rule (barycentric points, weights summing to 1)
};

// Directly stored coefficients of all lags of a set of edge pairs:
// for pair p = (i, j): lags m_lo .. m_lo+nlag-1 at val[off .. off+nlag).
struct PairStore {
  int64_t npairs = 0;
  int64_t nval = 0;
  int16_t* m_lo = nullptr;
  uint8_t* nlag = nullptr;
  int64_t* off = nullptr;   // [npairs]
  double* val = nullptr;    // [nval]; direct mode with one right-hand side: (hi, lo) FP32 pairs after setup
};

struct FmmPlan;

}  // namespace tdbem

struct tdbem_ctx {
  tdbem_params p;
  double dt = 0;
  int32_t Nt = 0;
  tdbem::Phys phys;
  int64_t nv = 0, nt = 0, ne = 0;
  double max_tri_rad = 0;            // max over triangles of centroid-vertex distance
  double max_quad_rad = 0;           // max over triangles of centroid-to-outer-rule-point distance
  // host mesh tables
  std::vector<double> V;
  std::vector<int32_t> T;
  std::vector<int32_t> ev, et, eo;  // [ne][2]
  std::vector<int32_t> te;          // [nt][3]
  std::vector<int8_t> ts;           // [nt][3]
  // device mesh
  tdbem::TriGeom tg{};
  int32_t* d_et = nullptr;          // [ne][2]
  // direct coefficients: rows i, all j (direct mode)
  tdbem::PairStore direct;
  tdbem::FmmPlan* fmm = nullptr;    // fast mode
  int32_t max_lag = 0;
  // Z0 in CSR
  int32_t* d_z0_ptr = nullptr;
  int32_t* d_z0_col = nullptr;
  double* d_z0_val = nullptr;
  double* d_z0_inv_diag = nullptr;
  float* d_z0_val32 = nullptr;
  float* d_z0_inv32 = nullptr;
  int64_t z0_nnz = 0;
  // the same Z0 as column-major ELL for the solver: entry k of row i at [k*ne + i]
  int32_t z0_ell_w = 0;             // largest row length
  int32_t* d_ell_len = nullptr;     // [ne]
  int32_t* d_ell_col = nullptr;     // [w][ne]
  double* d_ell_val = nullptr;      // [w][ne]
  float* d_ell_val32 = nullptr;     // [w][ne]
  int32_t* d_pc_col = nullptr;      // triangle-block preconditioner [5][ne] (precond = 1), else null
  float* d_pc_val = nullptr;
  // marching state; R right-hand sides share every operator and the RHS
  // index is the fastest one in every per-edge array ([..][ne][R]), so that
  // R = 1 is the plain single-RHS layout
  int32_t R = 1;                    // right-hand sides (params.n_rhs)
  int32_t L = 0;                    // ring length (power of two)
  double* d_Jring = nullptr;        // [ne][L][R]
  float2* d_ring2 = nullptr;        // direct mode, R = 1: split history [L][ne] (hi, lo) (untiled kernel)
  // direct mode, R = 1, tiled history sum (lags >= 3) plus the lag-2 entries in the reduction
  double* d_dpart = nullptr;        // partial sums [3][ncb][ne]: march steps alpha & 1, evaluations 2
  // direct mode, R = 1, row-tile store of the lags >= 3 (rows in tiles of 32,
  // one lane per row; see k_direct_history_rt)
  int32_t rt_prec = 0;              // 0: untiled (ring > 128 steps), 1: FP32 values, 2: (hi, lo) pairs, 3: 24-bit
  unsigned char* d_rt_val = nullptr;  // [groups] of 32 values (128, 256 or 96 bytes)
  uint32_t* d_rt_goff = nullptr;    // [nrt * ne + 1] first group of (tile, column)
  uint8_t* d_rt_lo = nullptr;       // [nrt * ne][32] first stored lag (>= 3) of (row, column)
  int32_t rt_Lh = 0;                // history rows staged per column (every lag a group reaches)
  int32_t rt_ncb = 0, rt_nrg = 0;   // column blocks and row-tile groups of its grid
  int32_t rt_tiles = 0;             // row tiles per block
  int64_t rt_bytes = 0;             // bytes streamed per launch (values, lag bytes, group offsets)
  int32_t* d_dt_err = nullptr;      // set by a bounded wait of the history sum that expired
  int64_t* d_l2_ptr = nullptr;      // lag-2 coefficients, CSR over rows [ne + 1]
  int32_t* d_l2_col = nullptr;
  double* d_l2_val = nullptr;
  cudaStream_t dstream = nullptr;   // far_overlap: the lags >= 3 of step alpha + 2 run here during step alpha + 1
  cudaEvent_t ev_dsolved = nullptr;
  cudaEvent_t ev_dahead[2] = {nullptr, nullptr};
  int32_t dahead[2] = {0, 0};       // step whose lags >= 3 sit in partial buffer b (0: none)
  double* d_R = nullptr;            // [ne][R]
  double* d_J = nullptr;            // [ne][R] current solution
  double* d_Vall = nullptr;         // [Nt-1][ne][R] or null
  double* d_pulse = nullptr;        // [R][10]
  double* d_stage = nullptr;        // [R][ne] host-layout staging (R > 1)
  bool have_pulse = false;
  std::vector<double> pulse;        // [R][10]
  double* d_work = nullptr;         // solver vectors [8][ne][R]
  double* d_dots = nullptr;         // solver reductions
  int32_t* d_status = nullptr;      // solver status / iterations [8]
  // asynchronous steps (tdbem_step_v_async / tdbem_step_wait): per slot the
  // step's solver status copied to pinned host memory and an event after its
  // copies; issued and waited counts
  static constexpr int kAsyncSlots = 4;
  int32_t* h_async_status = nullptr;  // pinned [kAsyncSlots][2]
  cudaEvent_t ev_async[kAsyncSlots] = {};
  int64_t async_issued = 0, async_waited = 0;
  int32_t alpha = 1;
  int64_t total_iters = 0;
  int64_t total_sweeps = 0;
  int32_t cluster = 0;              // CTAs of the single-RHS solve (one cluster, or the cooperative grid)
  double* d_gslots = nullptr;       // per-block partial sums of the grid-wide solve
  int32_t device = 0;               // CUDA device the context lives on
  double* d_Vtab = nullptr;         // [Nt-1][ne][R] incident field of every step (precomputed)
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  double setup_seconds = 0;
  int64_t device_bytes = 0;
  int64_t peak_bytes = 0;           // the most device_bytes has been
  // kernel-class timing (tdbem_profile_*)
  static constexpr int kClasses = 11;
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_marks;
  size_t ev_next = 0;
  cudaEvent_t prof_begin(int cls);
  void prof_end(int cls, cudaEvent_t b);
  std::string err;
  void set_error(const std::string& s) { err = s; }
  template <class T>
  tdbem_status dalloc(T** ptr, size_t count) {
    if (count == 0) count = 1;
    if (p.max_device_bytes > 0 && device_bytes + (int64_t)(count * sizeof(T)) > p.max_device_bytes) {
      set_error("device memory budget (max_device_bytes) exceeded");
      *ptr = nullptr;
      return TDBEM_ENOMEM;
    }
    cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
    if (e != cudaSuccess) {
      set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      *ptr = nullptr;
      return TDBEM_ENOMEM;
    }
    device_bytes += (int64_t)(count * sizeof(T));
    peak_bytes = std::max(peak_bytes, device_bytes);
    allocs.push_back((void*)*ptr);
    alloc_bytes.push_back(count * sizeof(T));
    return TDBEM_OK;
  }
  // returns an allocation of dalloc early (no-op for a pointer it did not make)
  void dfree(void* ptr) {
    for (size_t k = 0; k < allocs.size(); ++k)
      if (allocs[k] == ptr) {
        cudaFree(ptr);
        device_bytes -= (int64_t)alloc_bytes[k];
        allocs.erase(allocs.begin() + k);
        alloc_bytes.erase(alloc_bytes.begin() + k);
        return;
      }
  }
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;
  // learned warm start (mlp.cu)
  struct Mlp* mlp = nullptr;
};

// mesh.cu
tdbem_status tdbem_build_mesh(tdbem_ctx* c, const double* verts, int64_t nv, const int32_t* tris, int64_t ntri);
// direct.cu
tdbem_status tdbem_build_direct(tdbem_ctx* c);
tdbem_status tdbem_direct_history(tdbem_ctx* c, int32_t alpha, const double* d_ring, const double* V);
tdbem_status tdbem_direct_split(tdbem_ctx* c);
tdbem_status tdbem_direct_after_solve(tdbem_ctx* c, int32_t alpha);
tdbem_status tdbem_direct_join(tdbem_ctx* c);
tdbem_status tdbem_direct_check(tdbem_ctx* c);
tdbem_status tdbem_direct_invalidate(tdbem_ctx* c);
void tdbem_direct_free(tdbem_ctx* c);
tdbem_status tdbem_incident_table(tdbem_ctx* c, int32_t r);
const double* tdbem_incident_row(const tdbem_ctx* c, int32_t alpha);
tdbem_status tdbem_assemble_csr(tdbem_ctx* c, const int2* d_pairs, int64_t npairs, const int64_t* d_row_ptr,
                                const int32_t* d_col, int64_t nnz, int16_t** m_lo, uint8_t** nlag, int64_t** off,
                                double** val, int64_t* nval);
// fmm.cu
tdbem_status tdbem_build_fast(tdbem_ctx* c);
tdbem_status tdbem_fast_history(tdbem_ctx* c, int32_t alpha, const double* ring, const double* V, bool eval);
tdbem_status tdbem_fast_after_solve(tdbem_ctx* c, int32_t alpha);
tdbem_status tdbem_fast_replay_step(tdbem_ctx* c, int32_t alpha, const double* ring);
tdbem_status tdbem_fast_consume_eval_slot(tdbem_ctx* c, int32_t alpha);
tdbem_status tdbem_fast_eval_reset(tdbem_ctx* c);
tdbem_status tdbem_fast_reset(tdbem_ctx* c);
void tdbem_fast_free(tdbem_ctx* c);
tdbem_status tdbem_fast_join(tdbem_ctx* c);
tdbem_status tdbem_fast_invalidate(tdbem_ctx* c);
tdbem_status tdbem_fast_check(tdbem_ctx* c);
// m2l_tc.cu
// pC: each pair's (source cell, symmetry) combination; pk: the packed
// moments of tdbem_m2l_pack for this event
tdbem_status tdbem_m2l_tc(tdbem_ctx* c, int mt, const int4* gemm, const int4* tiles, int ntiles, const uint4* img, int P,
                          int pt, int PS, const int32_t* pO, const int32_t* pC, const int16_t* psym,
                          const int16_t* smap, const float* pk, int k, float* loc, int Q, int R, int prec,
                          const float* opinv, const float* pkinv, int32_t* err);
// pkinv: the FP16 form's per-row inverse scales (null for the other forms)
tdbem_status tdbem_m2l_pack(tdbem_ctx* c, const int32_t* cS, const int16_t* csym, int ncombo, const int16_t* smap,
                            const float* mom, int k, int R, int PS, int pt, float* pk, float* pkinv);
tdbem_status tdbem_m2l_tc_images(tdbem_ctx* c, const float* ops, int nop, int P, int prec, uint4** img,
                                 float** opinv);
// the FP16 form with the operator rows resident in shared memory (P <= 256):
// units [u0, u0 + n) of the level's list, and the FP16 hi/lo moment pack it reads
tdbem_status tdbem_m2l_res(tdbem_ctx* c, const int4* gemm, const int4* units, int u0, int n, const uint4* img, int P,
                           int pt, int PS, const int32_t* pO, const int32_t* pC, const int16_t* psym,
                           const int16_t* smap, const __half* pk16, int k, float* loc, int Q, int R,
                           const float* opinv, const float* pkinv, int32_t* err, int max_ctas);
tdbem_status tdbem_m2l_pack_f16(tdbem_ctx* c, const int32_t* cS, const int16_t* csym, int ncombo,
                                const int16_t* smap, const float* mom, int k, int R, int PS, int pt, __half* pk16,
                                float* pkinv);
void tdbem_fast_info(const tdbem_ctx* c, tdbem_info* info);
void tdbem_fast_state(tdbem_ctx* c, std::vector<std::pair<void*, size_t>>* bufs);
tdbem_status tdbem_fast_z0_source(const tdbem_ctx* c, const int64_t** row_ptr, const int32_t** col,
                                  const int16_t** m_lo, const uint8_t** nlag, const int64_t** off, const double** val);
// gemm_tc.cu: C (M x N, FP32) = or += A (M x K) . B (N x K)^T, BF16 row-major operands on the tensor cores
tdbem_status tdbem_gemm_bf16(tdbem_ctx* c, cudaStream_t st, const __nv_bfloat16* A, int64_t lda,
                             const __nv_bfloat16* B, int64_t ldb, float* C, int64_t ldc, int M, int N, int K, int add,
                             int ksplit, int32_t* err);
// mlp.cu
tdbem_status tdbem_mlp_before_solve(tdbem_ctx* c, int32_t alpha, int32_t* warm);
tdbem_status tdbem_mlp_after_solve(tdbem_ctx* c, int32_t alpha);
void tdbem_mlp_free(tdbem_ctx* c);
// solve.cu
tdbem_status tdbem_build_z0(tdbem_ctx* c);
tdbem_status tdbem_build_z0_csr(tdbem_ctx* c);
tdbem_status tdbem_solve_z0(tdbem_ctx* c, int32_t alpha, int32_t* iters, int32_t warm);
