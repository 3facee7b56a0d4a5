// capi.cu -- the extern "C" entry points of include/tdbem.h and the marching
// driver (paper Program 1).
#include <chrono>
#include <cmath>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "internal.h"

using namespace tdbem;

cudaEvent_t tdbem_ctx::prof_begin(int) {
  if (!prof_on) return nullptr;
  if (ev_next >= ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    ev_pool.push_back(e);
  }
  cudaEvent_t e = ev_pool[ev_next++];
  cudaEventRecord(e, stream);
  return e;
}

void tdbem_ctx::prof_end(int cls, cudaEvent_t b) {
  if (!prof_on || !b) return;
  if (ev_next >= ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    ev_pool.push_back(e);
  }
  cudaEvent_t e = ev_pool[ev_next++];
  cudaEventRecord(e, stream);
  prof_marks.push_back({cls, {b, e}});
}

// Checkpoint file helpers (tdbem_save, tdbem_load).
namespace {
constexpr char kCkMagic[8] = {'T', 'D', 'B', 'E', 'M', 'C', 'K', '1'};

struct CkHeader {
  int32_t mode, n_rhs, L, Nt, alpha, p_s, p_t, n_leaf, far_kernel, m2l_prec, nbuf;
  int32_t interp;  // s_interp | t_interp << 1 | a_deriv << 2 (0: the defaults)
  int64_t ne, nt;
  double dt, theta, zeta, chi;
  uint64_t mesh_hash;  // FNV-1a of the vertex and triangle arrays
};

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

CkHeader ck_header(const tdbem_ctx* c, int32_t nbuf) {
  CkHeader h;
  std::memset(&h, 0, sizeof(h));
  h.mode = c->p.mode;
  h.n_rhs = c->R;
  h.L = c->L;
  h.Nt = c->Nt;
  h.alpha = c->alpha;
  h.p_s = c->p.p_s;
  h.p_t = c->p.p_t;
  h.n_leaf = c->p.n_leaf;
  h.far_kernel = c->p.far_kernel;
  h.interp = c->p.s_interp | c->p.t_interp << 1 | c->p.a_deriv << 2;
  h.m2l_prec = c->p.m2l_prec;
  h.nbuf = nbuf;
  h.ne = c->ne;
  h.nt = c->nt;
  h.dt = c->dt;
  h.theta = c->p.theta;
  h.zeta = c->p.zeta;
  h.chi = c->p.chi;
  uint64_t x = 1469598103934665603ull;
  x = fnv1a(x, c->V.data(), c->V.size() * sizeof(double));
  x = fnv1a(x, c->T.data(), c->T.size() * sizeof(int32_t));
  h.mesh_hash = x;
  return h;
}

// the march state's device buffers: history ring, current solution, and in
// fast mode the far field's moments, local coefficients and far RHS ring
std::vector<std::pair<void*, size_t>> ck_buffers(tdbem_ctx* c) {
  const size_t NR = (size_t)c->ne * c->R;
  std::vector<std::pair<void*, size_t>> b = {{c->d_Jring, NR * c->L * sizeof(double)},
                                             {c->d_J, NR * sizeof(double)}};
  if (c->p.mode == TDBEM_FAST) tdbem_fast_state(c, &b);
  return b;
}
}  // namespace

extern "C" {

void tdbem_default_params(tdbem_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->d = 2;
  p->p_s = 4;
  p->p_t = 4;
  p->n_leaf = 64;
  p->theta = 1.0;
  p->zeta = 1.0;
  p->eps = 1.0;
  p->mu = 1.0;
  p->s_jump = 1.0;
  p->mode = TDBEM_DIRECT;
  p->p2p_prec = TDBEM_P_FP64;
  p->m2l_prec = TDBEM_P_FP32;
  p->solve_tol = 1e-13;
  p->solve_maxit = 1000;
  p->warm_start = 1;
  p->n_rhs = 1;
  p->jacobi_sweeps = 0;
  p->precond = 1;
  p->far_overlap = 1;
  p->solve_grid = 0;
  p->chi = 1.0;
}

static void fill_phys(tdbem_ctx* c) {
  Phys& ph = c->phys;
  ph.dt = c->dt;
  ph.eps = c->p.eps;
  ph.mu = c->p.mu;
  ph.c = 1.0 / std::sqrt(ph.eps * ph.mu);
  ph.eta = std::sqrt(ph.mu / ph.eps);
  ph.a = ph.c * c->dt;
  ph.theta = c->p.theta;
  ph.zeta = c->p.zeta;
  ph.chi = c->p.chi;
  ph.s_jump = c->p.s_jump;
  // 7-point degree-5 rule on the triangle (Radon): centroid and two orbits of 3
  const double r15 = std::sqrt(15.0);
  const double b1 = (6.0 - r15) / 21.0, b2 = (6.0 + r15) / 21.0;
  const double w0 = 9.0 / 40.0, w1 = (155.0 - r15) / 1200.0, w2 = (155.0 + r15) / 1200.0;
  const double pts[kNq][3] = {{1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0}, {b1, b1, 1 - 2 * b1}, {b1, 1 - 2 * b1, b1},
                              {1 - 2 * b1, b1, b1},              {b2, b2, 1 - 2 * b2}, {b2, 1 - 2 * b2, b2},
                              {1 - 2 * b2, b2, b2}};
  const double wts[kNq] = {w0, w1, w1, w1, w2, w2, w2};
  std::memcpy(ph.qb, pts, sizeof(pts));
  std::memcpy(ph.qw, wts, sizeof(wts));
}

void tdbem_destroy(tdbem_ctx* c) {
  if (!c) return;
  tdbem_fast_join(c);
  tdbem_direct_join(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  tdbem_direct_free(c);
  if (c->h_async_status) cudaFreeHost(c->h_async_status);
  for (cudaEvent_t e : c->ev_async)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  tdbem_fast_free(c);
  tdbem_mlp_free(c);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

static tdbem_status finish_create(tdbem_ctx* c) {
  tdbem_status s;
  int32_t need = c->max_lag + 1;
  int32_t L = 8;
  while (L < need) L <<= 1;
  c->L = L;
  const int64_t NR = c->ne * (int64_t)c->R;
  if ((s = c->dalloc(&c->d_Jring, NR * L)) || (s = c->dalloc(&c->d_R, NR)) || (s = c->dalloc(&c->d_J, NR)) ||
      (s = c->dalloc(&c->d_pulse, 10 * (int64_t)c->R)) || (c->R > 1 && (s = c->dalloc(&c->d_stage, NR))))
    return s;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_Jring, 0, NR * L * sizeof(double), c->stream));
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_J, 0, NR * sizeof(double), c->stream));
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, 16 * sizeof(int32_t), c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return TDBEM_OK;
}

tdbem_status tdbem_create(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri, double dt, int32_t Nt,
                          const tdbem_params* params, tdbem_ctx** out) {
  if (!out) return TDBEM_EINVAL;
  *out = nullptr;
  if (!verts || !tris || !(dt > 0) || Nt < 2) return TDBEM_EINVAL;
  tdbem_params p;
  if (params)
    p = *params;
  else
    tdbem_default_params(&p);
  if (p.d != 2 || p.p_s < 2 || p.p_s > 8 || p.p_t < 2 || p.p_t > 8 || p.n_leaf < 1 || !(p.eps > 0) ||
      p.m2l_prec < TDBEM_P_FP32 || p.m2l_prec > TDBEM_P_F16X3 ||
      !(p.mu > 0) || !(p.theta >= 0) || !(p.chi >= 0) || !(p.solve_tol > 0) || p.solve_maxit < 1 || p.n_rhs < 1 ||
      p.n_rhs > TDBEM_MAX_RHS || p.jacobi_sweeps < 0 ||
      (p.m2l_tile_rows != 0 && p.m2l_tile_rows != 1 && p.m2l_tile_rows != 128 && p.m2l_tile_rows != 256) || p.precond < 0 ||
      p.precond > 1 || (p.far_overlap != 0 && p.far_overlap != 1) || p.solve_grid < 0 || p.solve_grid > 2 ||
      p.far_kernel < 0 || p.far_kernel > 3 || p.max_device_bytes < 0 || p.s_interp < 0 || p.s_interp > 1 ||
      p.t_interp < 0 || p.t_interp > 1 || p.a_deriv < 0 || p.a_deriv > 2 ||
      (p.solve_cluster != 0 && p.solve_cluster != 1 && p.solve_cluster != 2 && p.solve_cluster != 4 &&
       p.solve_cluster != 8 && p.solve_cluster != 16) ||
      (p.p2p_prec != TDBEM_P_FP64 && p.p2p_prec != TDBEM_P_FP32 && p.p2p_prec != TDBEM_P_FP24) ||
      (p.mode == TDBEM_DIRECT && p.p2p_prec != TDBEM_P_FP64 && p.n_rhs != 1) ||
      (p.mode != TDBEM_DIRECT && p.mode != TDBEM_FAST))
    return TDBEM_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  tdbem_ctx* c = new (std::nothrow) tdbem_ctx();
  if (!c) return TDBEM_ENOMEM;
  c->p = p;
  c->dt = dt;
  c->Nt = Nt;
  c->R = p.n_rhs;
  c->pulse.assign(10 * (size_t)c->R, 0.0);
  fill_phys(c);
  // the library's own stream takes the highest priority, so that the steps'
  // kernels are dispatched ahead of the deferred far-field products (which
  // run on a lowest-priority stream) whenever both wait for an SM
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  cudaError_t e = cudaStreamCreateWithPriority(&c->own_stream, cudaStreamNonBlocking, prio_hi);
  if (e != cudaSuccess) {
    delete c;
    return e == cudaErrorMemoryAllocation ? TDBEM_ENOMEM : TDBEM_ECUDA;
  }
  c->stream = c->own_stream;
  cudaGetDevice(&c->device);
  tdbem_status s = tdbem_build_mesh(c, verts, nv, tris, ntri);
  if (!s) {
    if (p.mode == TDBEM_DIRECT) {
      s = tdbem_build_direct(c);
      if (!s) s = tdbem_build_z0(c);
    } else {
      s = tdbem_build_fast(c);
      if (!s) s = tdbem_build_z0_csr(c);
    }
  }
  if (!s) s = finish_create(c);
  if (!s && p.mode == TDBEM_DIRECT) s = tdbem_direct_split(c);
  if (s) {
    tdbem_destroy(c);
    return s;
  }
  c->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = c;
  return TDBEM_OK;
}

tdbem_status tdbem_num_edges(const tdbem_ctx* c, int64_t* ne) {
  if (!c || !ne) return TDBEM_EINVAL;
  *ne = c->ne;
  return TDBEM_OK;
}

tdbem_status tdbem_edges(const tdbem_ctx* c, int32_t* edge_vert, int32_t* edge_tri) {
  if (!c) return TDBEM_EINVAL;
  if (edge_vert) std::memcpy(edge_vert, c->ev.data(), 2 * c->ne * sizeof(int32_t));
  if (edge_tri) std::memcpy(edge_tri, c->et.data(), 2 * c->ne * sizeof(int32_t));
  return TDBEM_OK;
}

tdbem_status tdbem_set_stream(tdbem_ctx* c, void* stream) {
  if (!c) return TDBEM_EINVAL;
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->stream = stream ? (cudaStream_t)stream : c->own_stream;
  return TDBEM_OK;
}

tdbem_status tdbem_set_incident_plane(tdbem_ctx* c, int32_t rhs, const double* pulse) {
  if (!c || !pulse || rhs < 0 || rhs >= c->R) return TDBEM_EINVAL;
  if (!(pulse[7] > 0) && !(pulse[7] < 0 && pulse[6] > 0)) return TDBEM_EINVAL;
  double* hp = c->pulse.data() + 10 * (size_t)rhs;
  std::memcpy(hp, pulse, 10 * sizeof(double));
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_pulse + 10 * rhs, hp, 10 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  cudaEvent_t e = c->prof_begin(0);
  tdbem_status s = tdbem_incident_table(c, rhs);
  c->prof_end(0, e);
  if (s) return s;
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->have_pulse = true;
  return TDBEM_OK;
}

// y[i*R + r] = x[i] for i < n (one column of an [n][R] array)
__global__ void k_put_column(const double* x, int64_t n, int32_t R, int32_t r, double* y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i * R + r] = x[i];
}

// [ne][R] (device layout) -> [R][ne] (host layout) and back
__global__ void k_to_host_layout(const double* x, int64_t ne, int32_t R, double* y) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ne * R) return;
  int64_t i = t / R;
  int32_t r = (int32_t)(t - i * R);
  y[(int64_t)r * ne + i] = x[t];
}

__global__ void k_from_host_layout(const double* y, int64_t ne, int32_t R, double* x) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ne * R) return;
  int64_t i = t / R;
  int32_t r = (int32_t)(t - i * R);
  x[t] = y[(int64_t)r * ne + i];
}

static tdbem_status to_host_layout(tdbem_ctx* c, const double* x, double* y) {
  const int64_t n = c->ne * (int64_t)c->R;
  k_to_host_layout<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(x, c->ne, c->R, y);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}

static tdbem_status from_host_layout(tdbem_ctx* c, const double* y, double* x) {
  const int64_t n = c->ne * (int64_t)c->R;
  k_from_host_layout<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(y, c->ne, c->R, x);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}

tdbem_status tdbem_set_rhs(tdbem_ctx* c, int32_t rhs, const double* V) {
  if (!c || !V || rhs < 0 || rhs >= c->R) return TDBEM_EINVAL;
  tdbem_status s;
  const int64_t n = (int64_t)(c->Nt - 1) * c->ne;
  if (!c->d_Vall) {
    if ((s = c->dalloc(&c->d_Vall, n * c->R))) return s;
    TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_Vall, 0, n * c->R * sizeof(double), c->stream));
  }
  if (c->R == 1) {
    TDBEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_Vall, V, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  } else {
    double* tmp = nullptr;
    TDBEM_CUDA_TRY(c, cudaMallocAsync(&tmp, n * sizeof(double), c->stream));
    cudaError_t e = cudaMemcpyAsync(tmp, V, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
      k_put_column<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(tmp, n, c->R, rhs, c->d_Vall);
      e = cudaGetLastError();
    }
    cudaFreeAsync(tmp, c->stream);
    TDBEM_CUDA_TRY(c, e);
  }
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return TDBEM_OK;
}

// R^{alpha-1} = V^{alpha-1} - history (eq. R), ring holds the history.
// skip_rhs: R already holds V^{alpha-1}.
static tdbem_status eval_R(tdbem_ctx* c, int32_t alpha, const double* d_ring, bool skip_rhs = false,
                           bool eval = false) {
  const double* V = skip_rhs ? c->d_R : tdbem_incident_row(c, alpha);
  if (c->p.mode == TDBEM_FAST) return tdbem_fast_history(c, alpha, d_ring, V, eval);
  return tdbem_direct_history(c, alpha, d_ring, V);
}

// ring[(j*L + slot)*R + r] = x[r*ne + j] (x in the host layout [R][ne])
__global__ void k_ring_put(const double* x, int64_t ne, int32_t R, int32_t L, int32_t slot, double* ring) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ne * R) return;
  int64_t r = t / ne, j = t - r * ne;
  ring[(j * L + slot) * R + r] = x[t];
}

// Fast-mode history evaluation: the far field of target alpha-1 depends on
// every earlier gating event, so the events of steps 1 .. alpha-1 are replayed
// on the supplied history in a separate evaluation state, feeding the ring one
// step at a time exactly as the march does.
static tdbem_status fast_history_eval(tdbem_ctx* c, int32_t alpha, const double* J_hist, int32_t n_hist,
                                      double* d_ring, double* d_buf) {
  const int64_t NR = c->ne * (int64_t)c->R;
  tdbem_status s = tdbem_fast_eval_reset(c);
  if (s) return s;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(d_ring, 0, NR * c->L * sizeof(double), c->stream));
  // an empty history leaves every moment zero: nothing to replay
  const int32_t a_last = n_hist > 0 ? alpha - 1 : 0;
  for (int32_t a = 1; a <= a_last; ++a) {
    int32_t b = a - 1;  // J^{a-1} becomes known after step a
    if (b < n_hist) {
      TDBEM_CUDA_TRY(c, cudaMemcpyAsync(d_buf, J_hist + (int64_t)b * NR, NR * sizeof(double), cudaMemcpyHostToDevice,
                                        c->stream));
    } else {
      TDBEM_CUDA_TRY(c, cudaMemsetAsync(d_buf, 0, NR * sizeof(double), c->stream));
    }
    k_ring_put<<<(unsigned)((NR + 255) / 256), 256, 0, c->stream>>>(d_buf, c->ne, c->R, c->L, b & (c->L - 1), d_ring);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    // the march consumes (clears) the far slot of target a-1 at step a
    if ((s = tdbem_fast_consume_eval_slot(c, a))) return s;
    if ((s = tdbem_fast_replay_step(c, a, d_ring))) return s;
  }
  return eval_R(c, alpha, d_ring, false, true);
}

// Copy the device right-hand side d_R ([ne][R]) to the caller's [R][ne] array.
static cudaError_t copy_out(tdbem_ctx* c, const double* d_x, double* h_out) {
  const int64_t NR = c->ne * (int64_t)c->R;
  if (c->R > 1) {
    if (to_host_layout(c, d_x, c->d_stage)) return cudaErrorLaunchFailure;
    d_x = c->d_stage;
  }
  return cudaMemcpyAsync(h_out, d_x, NR * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
}

__global__ void k_stage_to_ring(const double* staged, int32_t b0, int32_t nb, int64_t ne, int32_t R, int32_t L,
                                double* ring);

tdbem_status tdbem_history_eval(tdbem_ctx* c, int32_t alpha, const double* J_hist, int32_t n_hist, double* R_out) {
  if (!c || !R_out || alpha < 1 || alpha > c->Nt - 1 || n_hist < 0 || (n_hist > 0 && !J_hist)) return TDBEM_EINVAL;
  const int64_t NR = c->ne * (int64_t)c->R;
  const int32_t L = c->L;
  // steps of the history that reach step alpha: b0 .. b1
  const int32_t b0 = std::max(0, alpha - c->max_lag);
  const int32_t b1 = std::min(alpha - 2, n_hist - 1);
  const int32_t nb = b1 >= b0 ? b1 - b0 + 1 : 0;
  const int64_t nstage = c->p.mode == TDBEM_FAST ? NR : (int64_t)nb * NR;
  double* d_ring = nullptr;
  TDBEM_CUDA_TRY(c, cudaMallocAsync(&d_ring, (NR * L + std::max<int64_t>(nstage, 1)) * sizeof(double), c->stream));
  double* d_stage = d_ring + NR * L;
  cudaError_t e = cudaSuccess;
  tdbem_status s = TDBEM_OK;
  if (c->p.mode == TDBEM_FAST) {
    s = fast_history_eval(c, alpha, J_hist, n_hist, d_ring, d_stage);
  } else {
    e = cudaMemsetAsync(d_ring, 0, NR * L * sizeof(double), c->stream);
    if (e == cudaSuccess && nb > 0) {
      e = cudaMemcpyAsync(d_stage, J_hist + (int64_t)b0 * NR, nstage * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream);
      if (e == cudaSuccess) {
        k_stage_to_ring<<<(unsigned)((nstage + 255) / 256), 256, 0, c->stream>>>(d_stage, b0, nb, c->ne, c->R, L,
                                                                                 d_ring);
        e = cudaGetLastError();
      }
    }
    if (e == cudaSuccess) s = eval_R(c, alpha, d_ring);
  }
  if (e == cudaSuccess && !s) e = copy_out(c, c->d_R, R_out);
  cudaFreeAsync(d_ring, c->stream);
  cudaError_t e2 = cudaStreamSynchronize(c->stream);
  if (s) return s;
  if (e != cudaSuccess || e2 != cudaSuccess) {
    c->set_error(std::string("history_eval: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    return TDBEM_ECUDA;
  }
  return TDBEM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free history evaluation: the history is staged in a fixed static
// device array instead of a per-call allocation.
static __device__ __align__(256) double g_noalloc_scratch[TDBEM_NOALLOC_SCRATCH_DOUBLES];

// ring[(j*L + (b mod L))*R + r] = staged[((b - b0)*R + r)*ne + j] for b = b0 .. b0+nb-1
__global__ void k_stage_to_ring(const double* staged, int32_t b0, int32_t nb, int64_t ne, int32_t R, int32_t L,
                                double* ring) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nb * R * ne) return;
  int64_t kr = t / ne, j = t - kr * ne;
  int32_t k = (int32_t)(kr / R), r = (int32_t)(kr - (int64_t)k * R);
  ring[(j * L + ((b0 + k) & (L - 1))) * R + r] = staged[t];
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

extern "C" tdbem_status tdbem_history_eval_noalloc(tdbem_ctx* c, int32_t alpha, const double* J_hist, int32_t n_hist,
                                                   double* R_out) {
  if (!c || !R_out || alpha < 1 || alpha > c->Nt - 1 || n_hist < 0 || (n_hist > 0 && !J_hist)) return TDBEM_EINVAL;
  if (c->p.mode != TDBEM_DIRECT) {
    c->set_error("history_eval_noalloc: direct mode only");
    return TDBEM_EINVAL;
  }
  const int64_t ne = c->ne, NR = ne * c->R;
  const int32_t L = c->L;
  const int32_t b0 = std::max(0, alpha - c->max_lag);
  const int32_t b1 = std::min(alpha - 2, n_hist - 1);
  const int32_t nb = b1 >= b0 ? b1 - b0 + 1 : 0;
  if (NR * L + (int64_t)nb * NR > (int64_t)TDBEM_NOALLOC_SCRATCH_DOUBLES) {
    c->set_error("history_eval_noalloc: problem needs " + std::to_string(NR * L + (int64_t)nb * NR) +
                 " doubles of scratch, more than TDBEM_NOALLOC_SCRATCH_DOUBLES");
    return TDBEM_EINVAL;
  }
  int dev = -1;
  TDBEM_CUDA_TRY(c, cudaGetDevice(&dev));
  if (dev != c->device || dev < 0 || dev >= kMaxDevices) {
    c->set_error("history_eval_noalloc: the context's device must be current");
    return TDBEM_EINVAL;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        c->set_error(std::string("history_eval_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return TDBEM_ECUDA;
      }
      g_noalloc_ptr[dev] = (double*)p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  double* ring = scratch;
  double* staged = scratch + NR * L;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(ring, 0, NR * L * sizeof(double), c->stream));
  if (nb > 0) {
    TDBEM_CUDA_TRY(c, cudaMemcpyAsync(staged, J_hist + (int64_t)b0 * NR, (int64_t)nb * NR * sizeof(double),
                                      cudaMemcpyHostToDevice, c->stream));
    int64_t n = (int64_t)nb * NR;
    k_stage_to_ring<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(staged, b0, nb, ne, c->R, L, ring);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
  }
  tdbem_status s = eval_R(c, alpha, ring);
  if (s) return s;
  TDBEM_CUDA_TRY(c, copy_out(c, c->d_R, R_out));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return TDBEM_OK;
}

static tdbem_status step_async(tdbem_ctx* c, bool have_V = false) {
  if (c->alpha > c->Nt - 1) {
    c->set_error("step: all Nt-1 steps already taken");
    return TDBEM_ESTATE;
  }
  tdbem_status s = eval_R(c, c->alpha, c->d_Jring, have_V);
  if (s) return s;
  int32_t warm = c->p.warm_start ? 1 : 0;
  if ((s = tdbem_mlp_before_solve(c, c->alpha, &warm))) return s;
  cudaEvent_t e = c->prof_begin(2);
  s = tdbem_solve_z0(c, c->alpha, nullptr, warm);
  c->prof_end(2, e);
  if (s) return s;
  if ((s = tdbem_mlp_after_solve(c, c->alpha))) return s;
  if (c->p.mode == TDBEM_FAST && (s = tdbem_fast_after_solve(c, c->alpha))) return s;
  if (c->p.mode == TDBEM_DIRECT && (s = tdbem_direct_after_solve(c, c->alpha))) return s;
  c->alpha++;
  return TDBEM_OK;
}

tdbem_status tdbem_step(tdbem_ctx* c, double* J_out, int32_t* iters) {
  if (!c) return TDBEM_EINVAL;
  tdbem_status s = step_async(c);
  if (s) return s;
  int32_t h[2];
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(h, c->d_status, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  if (J_out) TDBEM_CUDA_TRY(c, copy_out(c, c->d_J, J_out));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (iters) *iters = h[0];
  c->total_iters += h[0];
  if (c->p.mode == TDBEM_FAST && (s = tdbem_fast_check(c))) return s;
  if (!h[1]) {
    if (c->p.mode == TDBEM_DIRECT && (s = tdbem_direct_check(c))) return s;
    c->set_error("step: Z0 solve missed the tolerance");
    return TDBEM_ENOCONV;
  }
  return TDBEM_OK;
}

tdbem_status tdbem_step_v(tdbem_ctx* c, const double* V, double* J_out, int32_t* iters) {
  if (!c || !V) return TDBEM_EINVAL;
  const int64_t NR = c->ne * (int64_t)c->R;
  if (c->R == 1) {
    TDBEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_R, V, NR * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  } else {
    TDBEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_stage, V, NR * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    tdbem_status s0 = from_host_layout(c, c->d_stage, c->d_R);
    if (s0) return s0;
  }
  tdbem_status s = step_async(c, true);
  if (s) return s;
  int32_t h[2];
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(h, c->d_status, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  if (J_out) TDBEM_CUDA_TRY(c, copy_out(c, c->d_J, J_out));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (iters) *iters = h[0];
  c->total_iters += h[0];
  if (c->p.mode == TDBEM_FAST && (s = tdbem_fast_check(c))) return s;
  if (!h[1]) {
    if (c->p.mode == TDBEM_DIRECT && (s = tdbem_direct_check(c))) return s;
    c->set_error("step: Z0 solve missed the tolerance");
    return TDBEM_ENOCONV;
  }
  return TDBEM_OK;
}

// Wait for the oldest outstanding asynchronous step and check its status.
tdbem_status tdbem_step_wait(tdbem_ctx* c, int32_t* iters) {
  if (!c) return TDBEM_EINVAL;
  if (iters) *iters = 0;
  if (c->async_waited == c->async_issued) return TDBEM_OK;
  const int slot = (int)(c->async_waited % tdbem_ctx::kAsyncSlots);
  TDBEM_CUDA_TRY(c, cudaEventSynchronize(c->ev_async[slot]));
  ++c->async_waited;
  const int32_t it = c->h_async_status[2 * slot], conv = c->h_async_status[2 * slot + 1];
  if (iters) *iters = it;
  c->total_iters += it;
  tdbem_status s;
  if (c->p.mode == TDBEM_FAST && (s = tdbem_fast_check(c))) return s;
  if (!conv) {
    if (c->p.mode == TDBEM_DIRECT && (s = tdbem_direct_check(c))) return s;
    c->set_error("step: Z0 solve missed the tolerance");
    return TDBEM_ENOCONV;
  }
  return TDBEM_OK;
}

tdbem_status tdbem_step_v_async(tdbem_ctx* c, const double* V, double* J_out) {
  if (!c || !V) return TDBEM_EINVAL;
  tdbem_status s;
  if (!c->h_async_status) {
    TDBEM_CUDA_TRY(c, cudaMallocHost(&c->h_async_status, 2 * tdbem_ctx::kAsyncSlots * sizeof(int32_t)));
    for (cudaEvent_t& e : c->ev_async) TDBEM_CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  if (c->async_issued - c->async_waited == tdbem_ctx::kAsyncSlots && (s = tdbem_step_wait(c, nullptr))) return s;
  const int slot = (int)(c->async_issued % tdbem_ctx::kAsyncSlots);
  const int64_t NR = c->ne * (int64_t)c->R;
  if (c->R == 1) {
    TDBEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_R, V, NR * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  } else {
    TDBEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_stage, V, NR * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if ((s = from_host_layout(c, c->d_stage, c->d_R))) return s;
  }
  if ((s = step_async(c, true))) return s;
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(c->h_async_status + 2 * slot, c->d_status, 2 * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, c->stream));
  if (J_out) TDBEM_CUDA_TRY(c, copy_out(c, c->d_J, J_out));
  TDBEM_CUDA_TRY(c, cudaEventRecord(c->ev_async[slot], c->stream));
  ++c->async_issued;
  return TDBEM_OK;
}

// Every outstanding asynchronous step waited for (their statuses checked).
static tdbem_status drain_async(tdbem_ctx* c) {
  tdbem_status first = TDBEM_OK;
  while (c->async_waited < c->async_issued) {
    tdbem_status s = tdbem_step_wait(c, nullptr);
    if (s && !first) first = s;
  }
  return first;
}

tdbem_status tdbem_profile_enable(tdbem_ctx* c, int32_t on) {
  if (!c) return TDBEM_EINVAL;
  tdbem_status s = tdbem_fast_join(c);
  if (!s) s = tdbem_direct_join(c);
  if (s) return s;
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->prof_on = on != 0;
  c->prof_marks.clear();
  c->ev_next = 0;
  return TDBEM_OK;
}

tdbem_status tdbem_profile_read(tdbem_ctx* c, int64_t* launches, double* ms, int32_t* n_classes) {
  if (!c || !launches || !ms) return TDBEM_EINVAL;
  tdbem_status s = tdbem_fast_join(c);
  if (!s) s = tdbem_direct_join(c);
  if (s) return s;
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < tdbem_ctx::kClasses; ++k) {
    launches[k] = 0;
    ms[k] = 0.0;
  }
  for (auto& m : c->prof_marks) {
    float t = 0.f;
    TDBEM_CUDA_TRY(c, cudaEventElapsedTime(&t, m.second.first, m.second.second));
    launches[m.first] += 1;
    ms[m.first] += t;
  }
  if (n_classes) *n_classes = tdbem_ctx::kClasses;
  return TDBEM_OK;
}

static tdbem_status check_misses(tdbem_ctx* c) {
  if (c->p.mode == TDBEM_FAST) {
    tdbem_status s = tdbem_fast_join(c);
  if (!s) s = tdbem_direct_join(c);
    if (s) return s;
    s = tdbem_fast_check(c);
    if (s) return s;
  } else {
    tdbem_status s = tdbem_direct_check(c);
    if (s) return s;
  }
  int32_t h[8];
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(h, c->d_status, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->total_iters = h[3];
  c->total_sweeps = h[7];
  if (h[2]) {
    c->set_error("march: " + std::to_string(h[2]) + " Z0 solves missed the tolerance");
    return TDBEM_ENOCONV;
  }
  return TDBEM_OK;
}

tdbem_status tdbem_march(tdbem_ctx* c, int32_t n_steps, double* J_all) {
  if (!c || n_steps < 0) return TDBEM_EINVAL;
  for (int32_t k = 0; k < n_steps; ++k) {
    tdbem_status s = step_async(c);
    if (s) return s;
    if (J_all) TDBEM_CUDA_TRY(c, copy_out(c, c->d_J, J_all + (int64_t)k * c->ne * c->R));
  }
  return check_misses(c);
}

// One step of the march, its current stored at step k of J_all_dev (device, may be null).
static tdbem_status step_dev(tdbem_ctx* c, int32_t k, double* J_all_dev) {
  tdbem_status s = step_async(c);
  if (s) return s;
  if (J_all_dev) {
    double* dst = J_all_dev + (int64_t)k * c->ne * c->R;
    if (c->R == 1) {
      TDBEM_CUDA_TRY(c, cudaMemcpyAsync(dst, c->d_J, c->ne * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    } else if ((s = to_host_layout(c, c->d_J, dst))) {
      return s;
    }
  }
  return TDBEM_OK;
}

tdbem_status tdbem_march_dev(tdbem_ctx* c, int32_t n_steps, double* J_all_dev) {
  if (!c || n_steps < 0) return TDBEM_EINVAL;
  for (int32_t k = 0; k < n_steps; ++k) {
    tdbem_status s = step_dev(c, k, J_all_dev);
    if (s) return s;
  }
  return check_misses(c);
}

tdbem_status tdbem_march_many(tdbem_ctx* const* ctxs, int32_t n, const int32_t* n_steps, double* const* J_all_dev,
                              int32_t* failed) {
  if (failed) *failed = -1;
  if (!ctxs || n < 1 || !n_steps) return TDBEM_EINVAL;
  int32_t rounds = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (!ctxs[i] || n_steps[i] < 0) return TDBEM_EINVAL;
    for (int32_t j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return TDBEM_EINVAL;
    rounds = std::max(rounds, n_steps[i]);
  }
  for (int32_t k = 0; k < rounds; ++k)
    for (int32_t i = 0; i < n; ++i) {
      if (k >= n_steps[i]) continue;
      tdbem_status s = step_dev(ctxs[i], k, J_all_dev ? J_all_dev[i] : nullptr);
      if (s) {
        if (failed) *failed = i;
        return s;
      }
    }
  for (int32_t i = 0; i < n; ++i) {
    tdbem_status s = check_misses(ctxs[i]);
    if (s) {
      if (failed) *failed = i;
      return s;
    }
  }
  return TDBEM_OK;
}

tdbem_status tdbem_reset(tdbem_ctx* c) {
  if (!c) return TDBEM_EINVAL;
  drain_async(c);  // the outstanding steps' statuses no longer matter
  tdbem_status s0 = tdbem_fast_invalidate(c);
  if (!s0) s0 = tdbem_direct_invalidate(c);
  if (s0) return s0;
  const int64_t NR = c->ne * (int64_t)c->R;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_Jring, 0, NR * c->L * sizeof(double), c->stream));
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_J, 0, NR * sizeof(double), c->stream));
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, 16 * sizeof(int32_t), c->stream));
  if (c->p.mode == TDBEM_FAST) {
    tdbem_status s = tdbem_fast_reset(c);
    if (s) return s;
  }
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->alpha = 1;
  c->total_iters = 0;
  c->total_sweeps = 0;
  return TDBEM_OK;
}

// ---------------------------------------------------------------------------
// Checkpoints: the march state written to a file and read back (helpers above
// the extern "C" block).


tdbem_status tdbem_save(tdbem_ctx* c, const char* path) {
  if (!c || !path) return TDBEM_EINVAL;
  tdbem_status s = drain_async(c);
  if (!s) s = tdbem_fast_join(c);
  if (!s) s = tdbem_direct_join(c);
  if (s) return s;
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const auto bufs = ck_buffers(c);
  const CkHeader h = ck_header(c, (int32_t)bufs.size());
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    c->set_error(std::string("save: cannot open ") + path + " for writing");
    return TDBEM_EINVAL;
  }
  bool ok = std::fwrite(kCkMagic, 1, 8, f) == 8 && std::fwrite(&h, sizeof(h), 1, f) == 1;
  std::vector<char> host;
  for (size_t k = 0; ok && k < bufs.size(); ++k) {
    const int64_t n = (int64_t)bufs[k].second;
    host.resize(bufs[k].second);
    cudaError_t e = cudaMemcpy(host.data(), bufs[k].first, bufs[k].second, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      std::fclose(f);
      c->set_error(std::string("save: ") + cudaGetErrorString(e));
      return TDBEM_ECUDA;
    }
    ok = std::fwrite(&n, sizeof(n), 1, f) == 1 && std::fwrite(host.data(), 1, host.size(), f) == host.size();
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) {
    c->set_error(std::string("save: write to ") + path + " failed");
    return TDBEM_EINVAL;
  }
  return TDBEM_OK;
}

tdbem_status tdbem_load(tdbem_ctx* c, const char* path) {
  if (!c || !path) return TDBEM_EINVAL;
  tdbem_status s = tdbem_fast_invalidate(c);
  if (!s) s = tdbem_direct_invalidate(c);
  if (s) return s;
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    c->set_error(std::string("load: cannot open ") + path);
    return TDBEM_EINVAL;
  }
  const auto bufs = ck_buffers(c);
  const CkHeader want = ck_header(c, (int32_t)bufs.size());
  char magic[8];
  CkHeader h;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkMagic, 8) == 0 &&
            std::fread(&h, sizeof(h), 1, f) == 1;
  if (!ok) {
    std::fclose(f);
    c->set_error("load: not a checkpoint of this library");
    return TDBEM_EINVAL;
  }
  CkHeader cmp = h;
  cmp.alpha = want.alpha;  // the step is what the checkpoint brings
  if (std::memcmp(&cmp, &want, sizeof(h)) != 0 || h.alpha < 1 || h.alpha > c->Nt) {
    std::fclose(f);
    c->set_error("load: the checkpoint was written by a context with another mesh, time axis or parameters");
    return TDBEM_EINVAL;
  }
  std::vector<std::vector<char>> host(bufs.size());
  for (size_t k = 0; ok && k < bufs.size(); ++k) {
    int64_t n = 0;
    ok = std::fread(&n, sizeof(n), 1, f) == 1 && n == (int64_t)bufs[k].second;
    if (!ok) break;
    host[k].resize(bufs[k].second);
    ok = std::fread(host[k].data(), 1, host[k].size(), f) == host[k].size();
  }
  std::fclose(f);
  if (!ok) {
    c->set_error(std::string("load: ") + path + " is truncated or does not match this context");
    return TDBEM_EINVAL;
  }
  // every size checked: now overwrite the state
  for (size_t k = 0; k < bufs.size(); ++k)
    TDBEM_CUDA_TRY(c, cudaMemcpy(bufs[k].first, host[k].data(), host[k].size(), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, 16 * sizeof(int32_t), c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->alpha = h.alpha;
  return TDBEM_OK;
}

tdbem_status tdbem_alpha(const tdbem_ctx* c, int32_t* alpha) {
  if (!c || !alpha) return TDBEM_EINVAL;
  *alpha = c->alpha;
  return TDBEM_OK;
}

tdbem_status tdbem_get_info(const tdbem_ctx* c, tdbem_info* info) {
  if (!c || !info) return TDBEM_EINVAL;
  std::memset(info, 0, sizeof(*info));
  info->ne = c->ne;
  info->n_tri = c->nt;
  info->n_near_pairs = c->direct.npairs;
  info->near_coef_bytes = c->direct.nval * (int64_t)sizeof(double);
  info->device_bytes_peak = c->peak_bytes;
  if (c->p.mode == TDBEM_DIRECT && c->R == 1)
    info->history_bytes = c->rt_bytes;
  info->device_bytes = c->device_bytes;
  info->setup_seconds = c->setup_seconds;
  info->total_solver_iters = c->total_iters;
  info->total_jacobi_sweeps = c->total_sweeps;
  info->z0_nnz = c->z0_nnz;
  info->solver_cluster = c->cluster;
  info->max_lag = c->max_lag;
  if (c->p.mode == TDBEM_FAST) tdbem_fast_info(c, info);
  return TDBEM_OK;
}

const char* tdbem_last_error(const tdbem_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
