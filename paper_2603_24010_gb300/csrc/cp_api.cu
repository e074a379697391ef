// cp_api.cu -- host side of the C ABI declared in include/cp.h.
//
// The context owns its device buffers (cudaMalloc at the first step call,
// once the particle counts are known), issues every kernel on the caller's
// stream, and replays a captured CUDA graph of `compact_every` step launches
// plus one removal launch whenever a call covers that many steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "cp_device.cuh"
#include "cp_gap2d.cuh"

namespace cpk {
size_t push_smem_bytes(int N, int precision);
size_t solve_smem_bytes(int N, int ctas);
cudaError_t solve_cluster_size(int precision, int N, int* ctas);
cudaError_t push_configure(int precision, size_t push_smem);
cudaError_t solve_configure(int precision, size_t solve_smem);
cudaError_t push_occupancy(int precision, size_t smem, int* blocks_per_sm);
cudaError_t push_launch(int precision, const Bufs& B, int grid, size_t smem, cudaStream_t st,
                        int do_push);
cudaError_t solve_launch(int precision, const Bufs& B, int ctas, size_t smem, cudaStream_t st,
                         int do_push, int mode, double tol);
cudaError_t compact_launch(int precision, const Bufs& B, int grid, cudaStream_t st);
cudaError_t fill_launch(int precision, void* p, int64_t n, double v, cudaStream_t st);
cudaError_t load_pairs_launch(int precision, void* xe, void* ue, void* xo, void* uo, uint32_t* id,
                              int64_t n, int N, double th_e, double th_i, uint64_t seed, cudaStream_t st);
cudaError_t source_table_launch(const DevParams* P, double* vs, int64_t rows, cudaStream_t st);
cudaError_t pack_predictor_launch(const float* params, PredNet* net, cudaStream_t st);
size_t push_ens_smem_bytes(int n_max, int precision, int E);
int ens_max_instances();
size_t abs_rec_ens_bytes();
cudaError_t push_ens_occupancy(int precision, int threads, size_t smem, int* per_sm);
cudaError_t push_ens_launch(int precision, int threads, int grid, size_t smem, const Bufs* Ball,
                            int E, int n_max, void* abs, int abs_cap, cudaStream_t st);
cudaError_t compact_ens_launch(int precision, const Bufs* Ball, int E, int grid, cudaStream_t st);
cudaError_t solve_ens_configure(int precision, size_t smem);
cudaError_t solve_ens_launch(int precision, const Bufs* Ball, int n_inst, size_t smem,
                             cudaStream_t st, int do_push, int mode, double tol);
cudaError_t status_ens_launch(const Bufs* Ball, int E, int* out, cudaStream_t st);
cudaError_t push2_occupancy(int* per_sm);
cudaError_t push2_launch(const DevParams* P, DevState* S, void* D, const void* D_host, void* abs,
                         int abs_cap, int grid, cudaStream_t st);
cudaError_t sort2_launch(DevState* S, void* D, int T, int s, int sms, cudaStream_t st);
cudaError_t solve2_fwd_launch(void* D, long long* G1, int Nx, int Ny, cudaStream_t st);
cudaError_t solve2_modes_launch(void* D, int Nx, int Ny, float c_rhs, const double* E64,
                                cudaStream_t st);
cudaError_t deposit2_level0_launch(DevState* S, const void* D, int sms, cudaStream_t st);
cudaError_t tables2_launch(void* D, int Ny, double r2, cudaStream_t st);
cudaError_t samples_launch(const DevParams* P, const cp_diag* hist, int64_t first, int64_t n,
                           float* X, float* Y, cudaStream_t st);
}  // namespace cpk

using cpk::kSpecies;

struct cp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
  cpk::DevParams hp{};
  cpk::DevParams* dP = nullptr;
  cpk::DevState* dS = nullptr;
  int precision = CP_FP64;
  int N = 0;
  size_t es = 8;
  int64_t cap_req[kSpecies] = {0, 0, 0};
  int64_t cap[kSpecies] = {0, 0, 0};
  void* buf_xi[2][kSpecies] = {};
  void* buf_u[2][kSpecies] = {};
  uint32_t* buf_id[2] = {nullptr, nullptr};
  long long* G = nullptr;
  long long* Glast = nullptr;
  void* Epair = nullptr;
  double* phi = nullptr;
  double* E64 = nullptr;
  cpk::AbsRec* abs = nullptr;
  cp_diag* hist = nullptr;
  int64_t hist_rows = 0;
  double* vs = nullptr;
  int grid = 0;
  int compact_grid = 0;   // removal kernel
  size_t smem = 0;        // push kernel
  size_t solve_smem = 0;  // solve kernel
  int solve_ctas = 8;     // CTAs in the solve's cluster
  bool initialized = false;
  int compact_every = 128;
  int since_compact = 0;
  int64_t max_steps = 0;
  double sigma0 = 0.0;
  bool ens_member = false;  // advanced by a cp_batch (its own absorbed-ion lists unused)
  // particles staged on the host until the first step
  std::vector<double> hx[kSpecies], hu[kSpecies];
  std::vector<uint32_t> hid;
  // initial plasma drawn on the device at the first step (cp_load_species)
  int64_t load_n = -1;  // pairs, or -1 when electrons and ions come from cp_set_particles
  double load_T = 0.0;
  uint64_t load_seed = 0;
  cpk::PredNet* net = nullptr;  // installed predictor network (device), or null
  cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};  // strict, weak, learned weak
  double gtol[3] = {0.0, 0.0, 0.0};
  int64_t launches = 0;
  bool timing = false;
  double t_ms[3] = {0.0, 0.0, 0.0};  // push, solve, removal
  int64_t t_n[3] = {0, 0, 0};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<double> last_step_ms;
};

namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? CP_OK : CP_ERR_CUDA; }

#define CP_TRY(expr)                       \
  do {                                     \
    const int _rc = (expr);                \
    if (_rc != CP_OK) return _rc;          \
  } while (0)
#define CP_CUDA(expr) CP_TRY(cuda_rc(expr))

int64_t round4(int64_t n) { return (n + 3) & ~int64_t(3); }

// --- Tesla transformer (Sec. 2.1, App. A): BDF2 of the loop equations ----
// Matrix of the level-n terms; coupled: loop 4 without its 1/C3 (the load
// capacitor's voltage is then phi_0, Sec. 2.4.2).
void tesla_matrix(const cp_tesla& q, double dt, bool coupled, double T[5][5]) {
  const double a = 3.0 / (2.0 * dt), b = 9.0 / (4.0 * dt * dt);
  const double r1 = a * q.R1, r2 = a * q.R2, r3 = a * q.R3, m = b * q.M;
  const double rows[5][5] = {
      {1.0 / q.C1 + r1, -r1, 0.0, 0.0, -r1},
      {-r1, r1 + r2 + b * q.L1, m, 0.0, r1},
      {0.0, m, b * q.L2 + r3, -r3, r3},
      {0.0, 0.0, -r3, r3 + (coupled ? 0.0 : 1.0 / q.C3), -r3},
      {-r1, r1, r3, -r3, r1 + r3 + 1.0 / q.C2}};
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) T[i][j] = rows[i][j];
}

// History terms c = H h of the same equations, h[5 k + i] = Q_i of level n-1-k.
void tesla_history(const cp_tesla& q, double dt, const double h[20], double c[5]) {
  double h1[5], h2[5];
  for (int i = 0; i < 5; ++i) {
    h1[i] = (4.0 * h[i] - h[5 + i]) / (2.0 * dt);
    h2[i] = (24.0 * h[i] - 22.0 * h[5 + i] + 8.0 * h[10 + i] - h[15 + i]) / (4.0 * dt * dt);
  }
  const double x1 = h1[0] - h1[1] - h1[4], x3 = h1[2] - h1[3] + h1[4];
  c[0] = q.R1 * x1;
  c[1] = -q.R1 * x1 + q.R2 * h1[1] + q.L1 * h2[1] + q.M * h2[2];
  c[2] = q.M * h2[1] + q.L2 * h2[2] + q.R3 * x3;
  c[3] = -q.R3 * x3;
  c[4] = -q.R1 * x1 + q.R3 * x3;
}

// X = T^{-1} B for a 5 x m right-hand side (Gaussian elimination, partial pivoting).
bool solve5(double T[5][5], double* B, int m) {
  for (int k = 0; k < 5; ++k) {
    int piv = k;
    for (int i = k + 1; i < 5; ++i)
      if (std::fabs(T[i][k]) > std::fabs(T[piv][k])) piv = i;
    if (!(std::fabs(T[piv][k]) > 0.0)) return false;
    if (piv != k) {
      for (int j = 0; j < 5; ++j) std::swap(T[k][j], T[piv][j]);
      for (int j = 0; j < m; ++j) std::swap(B[k * m + j], B[piv * m + j]);
    }
    for (int i = k + 1; i < 5; ++i) {
      const double f = T[i][k] / T[k][k];
      for (int j = k; j < 5; ++j) T[i][j] -= f * T[k][j];
      for (int j = 0; j < m; ++j) B[i * m + j] -= f * B[k * m + j];
    }
  }
  for (int i = 4; i >= 0; --i)
    for (int j = 0; j < m; ++j) {
      double s = B[i * m + j];
      for (int l = i + 1; l < 5; ++l) s -= T[i][l] * B[l * m + j];
      B[i * m + j] = s / T[i][i];
    }
  return true;
}

// The linear maps of the strict and weak Tesla solves (cpk::DevParams t_*).
bool tesla_setup(const cp_tesla& q, double dt, cpk::DevParams* P) {
  double H[5 * 21];  // columns: H e_j (j < 20), then e4
  for (int j = 0; j < 20; ++j) {
    double h[20] = {0.0}, c[5];
    h[j] = 1.0;
    tesla_history(q, dt, h, c);
    for (int i = 0; i < 5; ++i) H[i * 21 + j] = c[i];
  }
  for (int i = 0; i < 5; ++i) H[i * 21 + 20] = (i == 3) ? 1.0 : 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    double T[5][5], X[5 * 21];
    std::memcpy(X, H, sizeof(X));
    tesla_matrix(q, dt, pass == 0, T);
    if (!solve5(T, X, 21)) return false;
    for (int i = 0; i < 5; ++i) {
      for (int j = 0; j < 20; ++j) (pass == 0 ? P->t_Ps : P->t_Pw)[i][j] = X[i * 21 + j];
      (pass == 0 ? P->t_ws : P->t_ww)[i] = X[i * 21 + 20];
    }
  }
  for (int i = 0; i < 5; ++i) P->t_Q0[i] = 0.0;
  P->t_Q0[0] = q.C1 * q.V1;
  return true;
}

// macroparticle weight and the charge scales that follow from it
void set_weight(cpk::DevParams* P, double w) {
  P->weight = w;
  P->scale = P->e * P->weight / (P->area * P->dx * cpk::kFix);
  P->alpha = P->dx * P->dx * P->scale / P->eps0;
}

cpk::Bufs make_bufs(const cp_ctx* c) {
  cpk::Bufs B;
  B.P = c->dP;
  B.S = c->dS;
  B.G = c->G;
  B.Glast = c->Glast;
  B.Epair = c->Epair;
  B.phi = c->phi;
  B.E64 = c->E64;
  B.abs = c->abs;
  B.hist = c->hist;
  B.hist_rows = c->hist_rows;
  B.vs = c->vs;
  B.net = c->net;
  // a single FP32 gap evaluates the predictor in the next push's idle tail;
  // ensemble members and the 2D gap's mean keep it in the solve
  B.net_in_push = (c->precision == CP_FP32 && !c->ens_member) ? 1 : 0;
  return B;
}

void free_all(cp_ctx* c) {
  for (int b = 0; b < 2; ++b) {
    for (int s = 0; s < kSpecies; ++s) {
      cudaFree(c->buf_xi[b][s]);
      cudaFree(c->buf_u[b][s]);
      c->buf_xi[b][s] = c->buf_u[b][s] = nullptr;
    }
    cudaFree(c->buf_id[b]);
    c->buf_id[b] = nullptr;
  }
  cudaFree(c->G);
  cudaFree(c->Glast);
  cudaFree(c->Epair);
  cudaFree(c->phi);
  cudaFree(c->E64);
  cudaFree(c->abs);
  cudaFree(c->hist);
  cudaFree(c->vs);
  cudaFree(c->dP);
  cudaFree(c->dS);
  cudaFree(c->net);
  for (int m = 0; m < 3; ++m)
    if (c->gexec[m]) cudaGraphExecDestroy(c->gexec[m]);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
}

int alloc(void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return CP_ERR_OOM;
  }
  return CP_OK;
}

// Allocate the stores, upload the staged particles and solve level 0.
int initialize(cp_ctx* c, int mode, double tol) {
  const cpk::DevParams& P = c->hp;
  int64_t n[kSpecies];
  for (int s = 0; s < kSpecies; ++s) n[s] = static_cast<int64_t>(c->hx[s].size());
  if (c->load_n >= 0) n[CP_ELECTRONS] = n[CP_IONS] = c->load_n;
  const int64_t B = P.beam_per_step;
  const int64_t K = c->compact_every;
  const int64_t ions_ever = n[1] + B * c->max_steps;
  const int64_t def[kSpecies] = {round4(n[0]) + 4 * K + 64, round4(ions_ever) + 4 * K + 64,
                                 std::max<int64_t>(65536, round4(ions_ever + n[2]) + 4 * K + 64)};
  for (int s = 0; s < kSpecies; ++s) {
    c->cap[s] = round4(c->cap_req[s] > 0 ? c->cap_req[s] : def[s]);
    if (n[s] > c->cap[s]) return CP_ERR_CAPACITY;
    c->hp.cap[s] = c->cap[s];
  }
  for (int b = 0; b < 2; ++b) {
    for (int s = 0; s < kSpecies; ++s) {
      CP_TRY(alloc(&c->buf_xi[b][s], c->es * c->cap[s]));
      CP_TRY(alloc(&c->buf_u[b][s], c->es * c->cap[s]));
      CP_CUDA(cpk::fill_launch(c->precision, c->buf_xi[b][s], c->cap[s], -1.0, c->stream));
      CP_CUDA(cudaMemsetAsync(c->buf_u[b][s], 0, c->es * c->cap[s], c->stream));
    }
    CP_TRY(alloc(reinterpret_cast<void**>(&c->buf_id[b]), sizeof(uint32_t) * c->cap[1]));
  }
  // initial plasma drawn on the device, or upload in store precision
  if (c->load_n > 0) {
    const double dxl = P.dx, dtl = P.dt;
    const double th_e = std::sqrt(P.e * c->load_T / P.m_e) * dtl / dxl;
    const double th_i = std::sqrt(P.e * c->load_T / P.m_i) * dtl / dxl;
    CP_CUDA(cpk::load_pairs_launch(c->precision, c->buf_xi[0][CP_ELECTRONS], c->buf_u[0][CP_ELECTRONS],
                                   c->buf_xi[0][CP_IONS], c->buf_u[0][CP_IONS], c->buf_id[0], c->load_n,
                                   c->N, th_e, th_i, c->load_seed, c->stream));
  }
  for (int s = 0; s < kSpecies; ++s) {
    if (!n[s] || (c->load_n >= 0 && s != CP_SECONDARIES)) continue;
    if (c->precision == CP_FP32) {
      std::vector<float> fx(n[s]), fu(n[s]);
      for (int64_t k = 0; k < n[s]; ++k) {
        fx[k] = static_cast<float>(c->hx[s][k]);
        fu[k] = static_cast<float>(c->hu[s][k]);
      }
      CP_CUDA(cudaMemcpyAsync(c->buf_xi[0][s], fx.data(), 4 * n[s], cudaMemcpyHostToDevice, c->stream));
      CP_CUDA(cudaMemcpyAsync(c->buf_u[0][s], fu.data(), 4 * n[s], cudaMemcpyHostToDevice, c->stream));
      CP_CUDA(cudaStreamSynchronize(c->stream));
    } else {
      CP_CUDA(cudaMemcpyAsync(c->buf_xi[0][s], c->hx[s].data(), 8 * n[s], cudaMemcpyHostToDevice, c->stream));
      CP_CUDA(cudaMemcpyAsync(c->buf_u[0][s], c->hu[s].data(), 8 * n[s], cudaMemcpyHostToDevice, c->stream));
      CP_CUDA(cudaStreamSynchronize(c->stream));
    }
  }
  uint32_t id_base = 0;
  if (c->load_n >= 0) {
    id_base = static_cast<uint32_t>(c->load_n);  // ids 0..n_pairs-1
  } else if (n[1]) {
    CP_CUDA(cudaMemcpyAsync(c->buf_id[0], c->hid.data(), 4 * n[1], cudaMemcpyHostToDevice, c->stream));
    for (uint32_t v : c->hid) id_base = std::max<uint32_t>(id_base, v + 1u);
  }
  if (static_cast<double>(id_base) + static_cast<double>(B) * c->max_steps > 4294967295.0)
    return CP_ERR_ARG;  // ion ids must stay within uint32

  CP_TRY(alloc(reinterpret_cast<void**>(&c->G), sizeof(long long) * (c->N + 1)));
  CP_TRY(alloc(reinterpret_cast<void**>(&c->Glast), sizeof(long long) * (c->N + 1)));
  CP_TRY(alloc(&c->Epair, 2 * c->es * (c->N + 1)));
  CP_TRY(alloc(reinterpret_cast<void**>(&c->phi), sizeof(double) * (c->N + 1)));
  CP_TRY(alloc(reinterpret_cast<void**>(&c->E64), sizeof(double) * c->N));
  c->hist_rows = c->max_steps + 1;
  CP_TRY(alloc(reinterpret_cast<void**>(&c->hist), sizeof(cp_diag) * c->hist_rows));
  CP_CUDA(cudaMemsetAsync(c->G, 0, sizeof(long long) * (c->N + 1), c->stream));
  CP_CUDA(cudaMemsetAsync(c->Glast, 0, sizeof(long long) * (c->N + 1), c->stream));
  CP_CUDA(cudaMemsetAsync(c->Epair, 0, 2 * c->es * (c->N + 1), c->stream));
  CP_CUDA(cudaMemsetAsync(c->hist, 0, sizeof(cp_diag) * c->hist_rows, c->stream));

  // launch shape: persistent grid of resident push CTAs, one solve cluster
  c->smem = cpk::push_smem_bytes(c->N, c->precision);
  CP_CUDA(cpk::solve_cluster_size(c->precision, c->N, &c->solve_ctas));
  c->solve_smem = cpk::solve_smem_bytes(c->N, c->solve_ctas);
  CP_CUDA(cpk::push_configure(c->precision, c->smem));
  CP_CUDA(cpk::solve_configure(c->precision, c->solve_smem));
  int per_sm = 0, sms = 0;
  CP_CUDA(cpk::push_occupancy(c->precision, c->smem, &per_sm));
  CP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  if (per_sm < 1) return CP_ERR_ARG;
  c->grid = per_sm * sms;
  c->compact_grid = 2 * sms;
  c->hp.abs_cap = 4096;
  CP_TRY(alloc(reinterpret_cast<void**>(&c->abs),
               sizeof(cpk::AbsRec) * (c->ens_member ? size_t(1)
                                                    : static_cast<size_t>(c->grid) * c->hp.abs_cap)));
  CP_TRY(alloc(reinterpret_cast<void**>(&c->dP), sizeof(cpk::DevParams)));
  CP_CUDA(cudaMemcpyAsync(c->dP, &c->hp, sizeof(cpk::DevParams), cudaMemcpyHostToDevice, c->stream));
  CP_TRY(alloc(reinterpret_cast<void**>(&c->vs), sizeof(double) * (c->hist_rows + 1)));
  CP_CUDA(cpk::source_table_launch(c->dP, c->vs, c->hist_rows + 1, c->stream));

  cpk::DevState S;
  std::memset(&S, 0, sizeof(S));
  for (int s = 0; s < kSpecies; ++s) {
    S.xi[s] = c->buf_xi[0][s];
    S.u[s] = c->buf_u[0][s];
    S.xi_alt[s] = c->buf_xi[1][s];
    S.u_alt[s] = c->buf_u[1][s];
    S.n_alloc[s] = round4(n[s]);
    S.n_proc[s] = round4(n[s]);
    S.n_live[s] = n[s];
  }
  S.id = c->buf_id[0];
  S.id_alt = c->buf_id[1];
  S.sigma = c->sigma0;
  S.beam_id_base = id_base;
  for (int k = 0; k < 4; ++k)  // the circuit rests before t = 0
    for (int i = 0; i < 5; ++i) S.Qt[k][i] = c->hp.t_Q0[i];
  CP_TRY(alloc(reinterpret_cast<void**>(&c->dS), sizeof(cpk::DevState)));
  CP_CUDA(cudaMemcpyAsync(c->dS, &S, sizeof(S), cudaMemcpyHostToDevice, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  for (int s = 0; s < kSpecies; ++s) {
    std::vector<double>().swap(c->hx[s]);
    std::vector<double>().swap(c->hu[s]);
  }
  std::vector<uint32_t>().swap(c->hid);
  c->initialized = true;
  // deposit rho^0 and solve level 0
  const cpk::Bufs B0 = make_bufs(c);
  CP_CUDA(cpk::push_launch(c->precision, B0, c->grid, c->smem, c->stream, 0));
  CP_CUDA(cpk::solve_launch(c->precision, B0, c->solve_ctas, c->solve_smem, c->stream, 0, mode, tol));
  c->launches += 2;
  return CP_OK;
}

int read_status(cp_ctx* c) {
  int st = 0;
  CP_CUDA(cudaMemcpyAsync(&st, &c->dS->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  return st;
}

// Capture compact_every step launches plus one removal launch into a graph.
int build_graph(cp_ctx* c, int mode, double tol) {
  if (c->gexec[mode] && c->gtol[mode] == tol) return CP_OK;
  if (c->gexec[mode]) {
    cudaGraphExecDestroy(c->gexec[mode]);
    c->gexec[mode] = nullptr;
  }
  const cpk::Bufs B = make_bufs(c);
  cudaGraph_t g = nullptr;
  CP_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < c->compact_every && e == cudaSuccess; ++k) {
    e = cpk::push_launch(c->precision, B, c->grid, c->smem, c->cap_stream, 1);
    if (e == cudaSuccess) e = cpk::solve_launch(c->precision, B, c->solve_ctas, c->solve_smem, c->cap_stream, 1, mode, tol);
  }
  if (e == cudaSuccess) e = cpk::compact_launch(c->precision, B, c->compact_grid, c->cap_stream);
  const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return CP_ERR_CUDA;
  }
  const cudaError_t e3 = cudaGraphInstantiate(&c->gexec[mode], g, 0);
  cudaGraphDestroy(g);
  CP_CUDA(e3);
  c->gtol[mode] = tol;
  return CP_OK;
}

// Launch one kernel (0 = push, 1 = solve, 2 = removal) between two timing events.
int timed_launch(cp_ctx* c, int which, int mode, double tol, std::vector<std::pair<int, size_t>>* rec) {
  const size_t k = rec->size() * 2;
  while (c->ev_pool.size() < k + 2) {
    cudaEvent_t e;
    CP_CUDA(cudaEventCreate(&e));
    c->ev_pool.push_back(e);
  }
  CP_CUDA(cudaEventRecord(c->ev_pool[k], c->stream));
  const cpk::Bufs B = make_bufs(c);
  if (which == 0)
    CP_CUDA(cpk::push_launch(c->precision, B, c->grid, c->smem, c->stream, 1));
  else if (which == 1)
    CP_CUDA(cpk::solve_launch(c->precision, B, c->solve_ctas, c->solve_smem, c->stream, 1, mode, tol));
  else
    CP_CUDA(cpk::compact_launch(c->precision, B, c->compact_grid, c->stream));
  CP_CUDA(cudaEventRecord(c->ev_pool[k + 1], c->stream));
  rec->push_back({which, k});
  return CP_OK;
}

int do_steps_timed(cp_ctx* c, int mode, int32_t n_steps, double tol) {
  std::vector<std::pair<int, size_t>> rec;
  rec.reserve(3 * static_cast<size_t>(n_steps) + 2);
  for (int k = 0; k < n_steps; ++k) {
    CP_TRY(timed_launch(c, 0, mode, tol, &rec));
    CP_TRY(timed_launch(c, 1, mode, tol, &rec));
    c->launches += 2;
    if (++c->since_compact == c->compact_every) {
      CP_TRY(timed_launch(c, 2, mode, tol, &rec));
      c->launches += 1;
      c->since_compact = 0;
    }
  }
  CP_CUDA(cudaStreamSynchronize(c->stream));
  c->last_step_ms.clear();
  for (const auto& r : rec) {
    float ms = 0.f;
    CP_CUDA(cudaEventElapsedTime(&ms, c->ev_pool[r.second], c->ev_pool[r.second + 1]));
    c->t_ms[r.first] += ms;
    c->t_n[r.first] += 1;
    if (r.first == 0) c->last_step_ms.push_back(ms);
  }
  return CP_OK;
}

int do_steps(cp_ctx* c, int mode, int32_t n_steps, double tol) {
  if (!c || n_steps < 0 || !(tol > 0.0)) return CP_ERR_ARG;
  CP_CUDA(cudaSetDevice(c->device));
  c->launches = 0;
  if (!c->initialized) CP_TRY(initialize(c, mode, tol));
  int64_t level = 0;
  CP_CUDA(cudaMemcpyAsync(&level, &c->dS->level, sizeof(level), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  if (level + n_steps > c->max_steps) return CP_ERR_ARG;
  if (c->timing) {
    CP_TRY(do_steps_timed(c, mode, n_steps, tol));
    return read_status(c);
  }
  const cpk::Bufs B = make_bufs(c);
  int left = n_steps;
  while (left > 0) {
    if (c->since_compact == 0 && left >= c->compact_every) {
      CP_TRY(build_graph(c, mode, tol));
      CP_CUDA(cudaGraphLaunch(c->gexec[mode], c->stream));
      c->launches += 2 * c->compact_every + 1;
      left -= c->compact_every;
      continue;
    }
    CP_CUDA(cpk::push_launch(c->precision, B, c->grid, c->smem, c->stream, 1));
    CP_CUDA(cpk::solve_launch(c->precision, B, c->solve_ctas, c->solve_smem, c->stream, 1, mode, tol));
    c->launches += 2;
    --left;
    if (++c->since_compact == c->compact_every) {
      CP_CUDA(cpk::compact_launch(c->precision, B, c->compact_grid, c->stream));
      c->launches += 1;
      c->since_compact = 0;
    }
  }
  return read_status(c);
}

}  // namespace

extern "C" {

int cp_create(const cp_gap* gap, const cp_circuit* circ, const cp_see_beam* see, const cp_run* run,
              void* stream, cp_ctx** out) {
  if (!gap || !circ || !see || !run || !out) return CP_ERR_ARG;
  *out = nullptr;
  if (gap->n_cells < 2 || !(gap->d > 0) || !(run->dt > 0) || !(gap->weight > 0) ||
      !(gap->eps0 > 0) || !(gap->e > 0) || !(gap->m_e > 0) || !(gap->m_i > 0) ||
      (run->precision != CP_FP64 && run->precision != CP_FP32) ||
      (circ->kind != CP_CIRCUIT_SERIES_RLC && circ->kind != CP_CIRCUIT_OPEN &&
       circ->kind != CP_CIRCUIT_TESLA) ||
      see->beam_per_step < 0 || (see->beam_mode != 0 && see->beam_mode != 1) || run->max_steps < 0 ||
      !(see->gamma_max >= 0.0 && see->gamma_max <= 14.0) ||
      (see->count_law != CP_SEE_COUNT_BERNOULLI && see->count_law != CP_SEE_COUNT_POISSON) ||
      (see->energy_law != CP_SEE_ENERGY_MAXWELL && see->energy_law != CP_SEE_ENERGY_LOGNORMAL))
    return CP_ERR_ARG;
  if (see->energy_law == CP_SEE_ENERGY_LOGNORMAL &&
      (!std::isfinite(see->ln_mu) || !(see->ln_sigma >= 0.0) || !(see->ln_mu + 9.0 * see->ln_sigma < 600.0)))
    return CP_ERR_ARG;  // exp(mu + sigma z) stays finite for |z| < 9 (|z| <= 8.6 from 52-bit draws)
  if (circ->kind == CP_CIRCUIT_SERIES_RLC && (!(circ->C > 0) || !(circ->R >= 0) || !(circ->L >= 0) ||
                                              !(circ->R > 0 || circ->L > 0) || !(circ->tau > 0)))
    return CP_ERR_ARG;
  if (circ->kind == CP_CIRCUIT_TESLA) {
    const cp_tesla& q = circ->tesla;
    const double pos[8] = {q.R1, q.R2, q.R3, q.C1, q.C2, q.C3, q.L1, q.L2};
    for (double v : pos)
      if (!(v > 0) || !std::isfinite(v)) return CP_ERR_ARG;
    if (!(q.M >= 0) || !(q.M * q.M < q.L1 * q.L2) || !std::isfinite(q.V1)) return CP_ERR_ARG;
  }
  const double C_load = (circ->kind == CP_CIRCUIT_TESLA) ? circ->tesla.C3 : circ->C;
  if (!(gap->area > 0) && !(C_load > 0)) return CP_ERR_ARG;
  cp_ctx* c = new (std::nothrow) cp_ctx();
  if (!c) return CP_ERR_OOM;
  int smem_optin = 0;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) !=
          cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return CP_ERR_CUDA;
  }
  // the push keeps the field table and the node sums of the whole gap in
  // shared memory (1 KB left for its static variables)
  if (cpk::push_smem_bytes(gap->n_cells, run->precision) + 1024 > static_cast<size_t>(smem_optin)) {
    cudaStreamDestroy(c->cap_stream);
    delete c;
    return CP_ERR_ARG;
  }
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  c->precision = run->precision;
  c->es = (run->precision == CP_FP32) ? sizeof(float) : sizeof(double);
  c->N = gap->n_cells;
  c->compact_every = run->compact_every > 0 ? run->compact_every : 128;
  c->max_steps = run->max_steps > 0 ? run->max_steps : 100000;
  c->sigma0 = gap->sigma0;
  for (int s = 0; s < kSpecies; ++s) c->cap_req[s] = run->capacity[s];
  cpk::DevParams& P = c->hp;
  P.N = gap->n_cells;
  P.circuit = circ->kind;
  P.beam_per_step = see->beam_per_step;
  P.beam_mode = see->beam_mode;
  P.d = gap->d;
  P.dx = gap->d / static_cast<double>(gap->n_cells);
  P.dt = run->dt;
  P.area = gap->area > 0 ? gap->area : C_load * gap->d / gap->eps0;
  P.eps0 = gap->eps0;
  P.e = gap->e;
  P.m_e = gap->m_e;
  P.m_i = gap->m_i;
  P.weight = gap->weight;
  P.R = circ->R;
  P.L = circ->L;
  P.C = C_load;
  P.V0 = circ->V0;
  P.f = circ->f;
  P.tau = circ->tau > 0 ? circ->tau : 1.0;
  P.polarity = circ->polarity;
  P.gamma_coef = see->gamma_coef;
  P.gamma_max = see->gamma_max;
  P.E_ref_eV = see->E_ref_eV > 0 ? see->E_ref_eV : 1000.0;
  P.see_scale = see->scale;
  P.T_emit_eV = see->T_emit_eV;
  P.beam_E_eV = see->beam_E_eV;
  P.beam_Emin_eV = see->beam_Emin_eV;
  P.beam_Emax_eV = see->beam_Emax_eV;
  // the oracle's order of operations: (sqrt((2 E) e / m_i) dt) / dx, each rounded
  P.beam_ub = std::sqrt(2.0 * P.beam_E_eV * gap->e / gap->m_i) * run->dt / (gap->d / gap->n_cells);
  {  // uniform beam in the FP32 pushes: (sqrt(2 E e / m_i) dt / dx)^2 = E k, linear in the draw
    const double r = run->dt / (gap->d / gap->n_cells);
    const double k = 2.0 * gap->e / gap->m_i * r * r;
    P.beam_c0 = P.beam_Emin_eV * k;
    P.beam_c1 = (P.beam_Emax_eV - P.beam_Emin_eV) * k;
  }
  P.seed = run->seed;
  P.scale = P.e * P.weight / (P.area * P.dx * cpk::kFix);
  const double dt = P.dt, dx = P.dx;
  P.kappa[CP_ELECTRONS] = -P.e * dt * dt / (P.m_e * dx);
  P.kappa[CP_IONS] = P.e * dt * dt / (P.m_i * dx);
  P.kappa[CP_SECONDARIES] = P.kappa[CP_ELECTRONS];
  P.see_vth = std::sqrt(P.e * P.T_emit_eV / P.m_e);
  P.see_count_law = see->count_law;
  P.see_energy_law = see->energy_law;
  P.see_ln_mu = see->ln_mu;
  P.see_ln_sigma = see->ln_sigma;
  P.see_v_eV = std::sqrt(2.0 * P.e / P.m_e);
  P.a21 = 9.0 * P.L / (4.0 * dt * dt) + 3.0 * P.R / (2.0 * dt);
  P.alpha = dx * dx * P.scale / P.eps0;
  P.g_strict = P.a21 > 0 ? 1.0 / P.a21 : 0.0;
  P.g_weak = 1.0 / (P.a21 + 1.0 / P.C);
  P.inv_C = P.C > 0 ? 1.0 / P.C : 0.0;
  P.gam_strict = P.g_strict * dx / (P.eps0 * P.area);
  P.inv_den_strict = 1.0 / (1.0 + static_cast<double>(P.N) * P.gam_strict);
  P.dx_eps0 = dx / P.eps0;
  P.inv_A = 1.0 / P.area;
  P.inv_dx = 1.0 / dx;
  P.inv_2dt = 1.0 / (2.0 * dt);
  P.L4dt2 = P.L / (4.0 * dt * dt);
  P.R2dt = P.R / (2.0 * dt);
  for (int s = 0; s < kSpecies; ++s) {
    P.kap_d[0][s] = 0.5 * P.kappa[s];
    P.kap_d[1][s] = P.kappa[s];
    P.kap_f[0][s] = static_cast<float>(P.kap_d[0][s]);
    P.kap_f[1][s] = static_cast<float>(P.kap_d[1][s]);
  }
  P.precision = run->precision;
  if (circ->kind == CP_CIRCUIT_TESLA) {
    if (!tesla_setup(circ->tesla, dt, &P)) {
      cudaStreamDestroy(c->cap_stream);
      delete c;
      return CP_ERR_ARG;
    }
    P.gam_tesla = P.t_ws[3] * dx / (P.eps0 * P.area);
    P.inv_den_tesla = 1.0 / (1.0 + static_cast<double>(P.N) * P.gam_tesla);
    P.V0 = 0.0;  // no source: the circuit starts from the charged C1
  }
  *out = c;
  return CP_OK;
}

int cp_set_particles(cp_ctx* c, int32_t species, const double* x, const double* v,
                     const uint32_t* id, int64_t n, int32_t units) {
  if (!c || species < 0 || species >= kSpecies || n < 0 || c->initialized ||
      (units != CP_UNITS_CELL && units != CP_UNITS_SI) || (n > 0 && (!x || !v)) ||
      (c->load_n >= 0 && species != CP_SECONDARIES))
    return CP_ERR_ARG;
  if (c->cap_req[species] > 0 && n > c->cap_req[species]) return CP_ERR_CAPACITY;
  const double dx = c->hp.dx, dt = c->hp.dt;
  const double N = static_cast<double>(c->N);
  std::vector<double> hx(n), hu(n);
  for (int64_t k = 0; k < n; ++k) {
    double xi = units == CP_UNITS_SI ? x[k] / dx : x[k];
    double u = units == CP_UNITS_SI ? v[k] * dt / dx : v[k];
    if (!(xi > 0.0) || !(xi < N) || !std::isfinite(u)) return CP_ERR_ARG;
    if (c->precision == CP_FP32) {
      float f = static_cast<float>(xi);
      if (f >= static_cast<float>(N)) f = std::nextafter(static_cast<float>(N), 0.0f);
      if (!(f > 0.0f)) f = 1.17549435e-38f;
      xi = f;
      u = static_cast<float>(u);
    }
    hx[k] = xi;
    hu[k] = u;
  }
  c->hx[species].swap(hx);
  c->hu[species].swap(hu);
  if (species == CP_IONS) {
    c->hid.resize(n);
    for (int64_t k = 0; k < n; ++k) c->hid[k] = id ? id[k] : static_cast<uint32_t>(k);
  }
  return CP_OK;
}

int cp_load_species(cp_ctx* c, const cp_species* sp, uint64_t seed) {
  if (!c || !sp || c->initialized || sp->n_pairs < 0 || sp->n_pairs > 4294967295LL ||
      !(sp->T_load_eV >= 0.0) || !std::isfinite(sp->T_load_eV) || !(sp->n0 >= 0.0) ||
      !std::isfinite(sp->n0) || !(sp->weight >= 0.0) || !std::isfinite(sp->weight))
    return CP_ERR_ARG;
  for (int s = 0; s < 2; ++s)
    if (c->cap_req[s] > 0 && sp->n_pairs > c->cap_req[s]) return CP_ERR_CAPACITY;
  double w = 0.0;
  if (sp->weight > 0.0) w = sp->weight;
  else if (sp->n0 > 0.0 && sp->n_pairs > 0)
    w = sp->n0 * c->hp.d * c->hp.area / static_cast<double>(sp->n_pairs);
  if (w > 0.0) set_weight(&c->hp, w);
  for (int s = 0; s < 2; ++s) {
    std::vector<double>().swap(c->hx[s]);
    std::vector<double>().swap(c->hu[s]);
  }
  std::vector<uint32_t>().swap(c->hid);
  c->load_n = sp->n_pairs;
  c->load_T = sp->T_load_eV;
  c->load_seed = seed;
  return CP_OK;
}

int cp_step_strict(cp_ctx* c, int32_t n_steps, double residual_tol) {
  return do_steps(c, 0, n_steps, residual_tol);
}

int cp_step_weak(cp_ctx* c, int32_t n_steps) { return do_steps(c, 1, n_steps, 1e300); }

int cp_step_weak_learned(cp_ctx* c, int32_t n_steps) {
  if (!c || !c->net) return CP_ERR_ARG;
  return do_steps(c, 2, n_steps, 1e300);
}

int cp_set_predictor(cp_ctx* c, const float* params, const cp_predictor* norm) {
  if (!c || !params || !norm) return CP_ERR_ARG;
  for (int f = 0; f < CP_PRED_FEATURES; ++f)
    if (!(norm->in_scale[f] > 0.0f) || !std::isfinite(norm->in_scale[f])) return CP_ERR_ARG;
  for (int o = 0; o < CP_MLP_OUT; ++o)
    if (!(norm->out_scale[o] > 0.0f) || !std::isfinite(norm->out_scale[o])) return CP_ERR_ARG;
  if (!(norm->bound > 0.0) || !std::isfinite(norm->bound)) return CP_ERR_ARG;
  for (int k = 0; k < CP_MLP_NPARAM; ++k)
    if (!std::isfinite(params[k])) return CP_ERR_ARG;
  CP_CUDA(cudaSetDevice(c->device));
  if (!c->net) CP_TRY(alloc(reinterpret_cast<void**>(&c->net), cpk::kPredNetBytes));
  float* dparams = nullptr;
  CP_TRY(alloc(reinterpret_cast<void**>(&dparams), sizeof(float) * CP_MLP_NPARAM));
  int rc = cuda_rc(cudaMemcpyAsync(dparams, params, sizeof(float) * CP_MLP_NPARAM,
                                   cudaMemcpyHostToDevice, c->stream));
  if (rc == CP_OK) rc = cuda_rc(cpk::pack_predictor_launch(dparams, c->net, c->stream));
  // scales and bound go straight into the packed struct
  if (rc == CP_OK)
    rc = cuda_rc(cudaMemcpyAsync(c->net->in_scale, norm->in_scale, sizeof(norm->in_scale),
                                 cudaMemcpyHostToDevice, c->stream));
  if (rc == CP_OK)
    rc = cuda_rc(cudaMemcpyAsync(c->net->out_scale, norm->out_scale, sizeof(norm->out_scale),
                                 cudaMemcpyHostToDevice, c->stream));
  if (rc == CP_OK)
    rc = cuda_rc(cudaMemcpyAsync(&c->net->bound, &norm->bound, sizeof(double),
                                 cudaMemcpyHostToDevice, c->stream));
  double inv[CP_PRED_FEATURES];
  for (int f = 0; f < CP_PRED_FEATURES; ++f) inv[f] = 1.0 / static_cast<double>(norm->in_scale[f]);
  if (rc == CP_OK)
    rc = cuda_rc(cudaMemcpyAsync(c->net->inv_in_scale, inv, sizeof(inv), cudaMemcpyHostToDevice,
                                 c->stream));
  if (rc == CP_OK) rc = cuda_rc(cudaStreamSynchronize(c->stream));
  cudaFree(dparams);
  // graphs captured before carry the old buffer set: rebuild on next use
  for (int m = 0; m < 3; ++m) {
    if (c->gexec[m]) cudaGraphExecDestroy(c->gexec[m]);
    c->gexec[m] = nullptr;
  }
  return rc;
}

int cp_predictor_samples(cp_ctx* c, int64_t first_level, int64_t n, float* X, float* Y) {
  if (!c || !X || !Y || n < 0 || first_level < CP_PRED_WINDOW || !c->initialized) return CP_ERR_ARG;
  int64_t level = 0;
  CP_CUDA(cudaSetDevice(c->device));
  CP_CUDA(cudaMemcpyAsync(&level, &c->dS->level, sizeof(level), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  if (first_level + n > level || first_level + n >= c->hist_rows) return CP_ERR_ARG;
  if (n == 0) return CP_OK;
  CP_CUDA(cpk::samples_launch(c->dP, c->hist, first_level, n, X, Y, c->stream));
  return CP_OK;
}

int cp_read_scalars(cp_ctx* c, cp_diag* out) {
  if (!c || !out) return CP_ERR_ARG;
  if (!c->initialized) return CP_ERR_ARG;
  CP_CUDA(cudaMemcpyAsync(out, &c->dS->cur, sizeof(cp_diag), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  return CP_OK;
}

int cp_read_history(cp_ctx* c, int64_t first, int64_t n, cp_diag* out) {
  if (!c || !out || first < 0 || n < 0 || !c->initialized) return CP_ERR_ARG;
  int64_t level = 0;
  CP_CUDA(cudaMemcpyAsync(&level, &c->dS->level, sizeof(level), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  if (first + n > level + 1 || first + n > c->hist_rows) return CP_ERR_ARG;
  if (n == 0) return CP_OK;
  CP_CUDA(cudaMemcpyAsync(out, c->hist + first, sizeof(cp_diag) * n, cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  return CP_OK;
}

int cp_read_grid(cp_ctx* c, double* phi, double* rho, double* E, int64_t* G, int32_t n_nodes) {
  if (!c || n_nodes != c->N + 1 || !c->initialized) return CP_ERR_ARG;
  const int N = c->N;
  std::vector<long long> g(N + 1);
  if (phi) CP_CUDA(cudaMemcpyAsync(phi, c->phi, sizeof(double) * (N + 1), cudaMemcpyDeviceToHost, c->stream));
  if (E) CP_CUDA(cudaMemcpyAsync(E, c->E64, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaMemcpyAsync(g.data(), c->Glast, sizeof(long long) * (N + 1), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  for (int i = 0; i <= N; ++i) {
    if (G) G[i] = g[i];
    if (rho) rho[i] = static_cast<double>(g[i]) * c->hp.scale;
  }
  return CP_OK;
}

int cp_get_particles(cp_ctx* c, int32_t species, double* xi, double* u, uint32_t* id, int64_t cap,
                     int64_t* n) {
  if (!c || species < 0 || species >= kSpecies || !n) return CP_ERR_ARG;
  if (!c->initialized) {
    const int64_t m = static_cast<int64_t>(c->hx[species].size());
    *n = m;
    if (m > cap) return CP_ERR_CAPACITY;
    for (int64_t k = 0; k < m; ++k) {
      if (xi) xi[k] = c->hx[species][k];
      if (u) u[k] = c->hu[species][k];
      if (id && species == CP_IONS) id[k] = c->hid[k];
    }
    return CP_OK;
  }
  cpk::DevState S;
  CP_CUDA(cudaMemcpyAsync(&S, c->dS, sizeof(S), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  const int64_t slots = std::min<int64_t>(S.n_alloc[species], c->cap[species]);
  std::vector<unsigned char> bx(c->es * slots), bu(c->es * slots);
  std::vector<uint32_t> bi(species == CP_IONS ? slots : 0);
  if (slots) {
    CP_CUDA(cudaMemcpyAsync(bx.data(), S.xi[species], c->es * slots, cudaMemcpyDeviceToHost, c->stream));
    CP_CUDA(cudaMemcpyAsync(bu.data(), S.u[species], c->es * slots, cudaMemcpyDeviceToHost, c->stream));
    if (species == CP_IONS)
      CP_CUDA(cudaMemcpyAsync(bi.data(), S.id, 4 * slots, cudaMemcpyDeviceToHost, c->stream));
    CP_CUDA(cudaStreamSynchronize(c->stream));
  }
  int64_t m = 0;
  for (int64_t k = 0; k < slots; ++k) {
    double xv, uv;
    if (c->precision == CP_FP32) {
      xv = reinterpret_cast<const float*>(bx.data())[k];
      uv = reinterpret_cast<const float*>(bu.data())[k];
    } else {
      xv = reinterpret_cast<const double*>(bx.data())[k];
      uv = reinterpret_cast<const double*>(bu.data())[k];
    }
    if (!(xv > 0.0)) continue;
    if (m < cap) {
      if (xi) xi[m] = xv;
      if (u) u[m] = uv;
      if (id && species == CP_IONS) id[m] = bi[k];
    }
    ++m;
  }
  *n = m;
  return m > cap ? CP_ERR_CAPACITY : CP_OK;
}

int cp_get_level(cp_ctx* c, int64_t* level) {
  if (!c || !level) return CP_ERR_ARG;
  if (!c->initialized) {
    *level = 0;
    return CP_OK;
  }
  CP_CUDA(cudaMemcpyAsync(level, &c->dS->level, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  return CP_OK;
}

// ---- checkpoint ---------------------------------------------------------------
namespace {
constexpr uint64_t kMagic = 0x31504b434350ULL;  // "PCCKP1"
struct SaveHeader {
  uint64_t magic;
  int64_t N, precision, level, hist_n, since_compact;
  int64_t slots[kSpecies];
  int64_t cap[kSpecies];
};
}  // namespace

int cp_save_state(cp_ctx* c, void* buf, size_t* len) {
  if (!c || !len || !c->initialized) return CP_ERR_ARG;
  cpk::DevState S;
  CP_CUDA(cudaMemcpyAsync(&S, c->dS, sizeof(S), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  SaveHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kMagic;
  h.N = c->N;
  h.precision = c->precision;
  h.level = S.level;
  h.hist_n = std::min<int64_t>(S.level + 1, c->hist_rows);
  h.since_compact = c->since_compact;
  size_t need = sizeof(h) + sizeof(S);
  for (int s = 0; s < kSpecies; ++s) {
    h.slots[s] = S.n_alloc[s];
    h.cap[s] = c->cap[s];
    need += 2 * c->es * h.slots[s];
  }
  need += 4 * h.slots[1];
  need += 2 * c->es * (c->N + 1) + sizeof(double) * (2 * c->N + 1) + sizeof(long long) * (c->N + 1);
  need += sizeof(cp_diag) * h.hist_n;
  if (!buf) {
    *len = need;
    return CP_OK;
  }
  if (*len < need) return CP_ERR_ARG;
  unsigned char* p = static_cast<unsigned char*>(buf);
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  std::memcpy(p, &S, sizeof(S));
  p += sizeof(S);
  auto d2h = [&](const void* src, size_t bytes) -> int {
    if (bytes) CP_CUDA(cudaMemcpyAsync(p, src, bytes, cudaMemcpyDeviceToHost, c->stream));
    p += bytes;
    return CP_OK;
  };
  for (int s = 0; s < kSpecies; ++s) {
    CP_TRY(d2h(S.xi[s], c->es * h.slots[s]));
    CP_TRY(d2h(S.u[s], c->es * h.slots[s]));
  }
  CP_TRY(d2h(S.id, 4 * h.slots[1]));
  CP_TRY(d2h(c->Epair, 2 * c->es * (c->N + 1)));
  CP_TRY(d2h(c->phi, sizeof(double) * (c->N + 1)));
  CP_TRY(d2h(c->E64, sizeof(double) * c->N));
  CP_TRY(d2h(c->Glast, sizeof(long long) * (c->N + 1)));
  CP_TRY(d2h(c->hist, sizeof(cp_diag) * h.hist_n));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  *len = need;
  return CP_OK;
}

int cp_load_state(cp_ctx* c, const void* buf, size_t len) {
  if (!c || !buf || len < sizeof(SaveHeader) + sizeof(cpk::DevState)) return CP_ERR_ARG;
  SaveHeader h;
  const unsigned char* p = static_cast<const unsigned char*>(buf);
  std::memcpy(&h, p, sizeof(h));
  p += sizeof(h);
  if (h.magic != kMagic || h.N != c->N || h.precision != c->precision) return CP_ERR_ARG;
  if (!c->initialized) {
    // allocate with the saved capacities
    for (int s = 0; s < kSpecies; ++s) {
      c->cap_req[s] = h.cap[s];
      c->hx[s].clear();
      c->hu[s].clear();
    }
    c->hid.clear();
    CP_TRY(initialize(c, 0, 1e300));
  }
  for (int s = 0; s < kSpecies; ++s)
    if (h.slots[s] > c->cap[s]) return CP_ERR_CAPACITY;
  if (h.hist_n > c->hist_rows) return CP_ERR_CAPACITY;
  cpk::DevState saved, cur;
  std::memcpy(&saved, p, sizeof(saved));
  p += sizeof(saved);
  CP_CUDA(cudaMemcpyAsync(&cur, c->dS, sizeof(cur), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  // keep this context's buffers, take everything else from the checkpoint
  cpk::DevState S = saved;
  for (int s = 0; s < kSpecies; ++s) {
    S.xi[s] = cur.xi[s];
    S.u[s] = cur.u[s];
    S.xi_alt[s] = cur.xi_alt[s];
    S.u_alt[s] = cur.u_alt[s];
  }
  S.id = cur.id;
  S.id_alt = cur.id_alt;
  auto h2d = [&](void* dst, size_t bytes) -> int {
    if (bytes) CP_CUDA(cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, c->stream));
    p += bytes;
    return CP_OK;
  };
  for (int s = 0; s < kSpecies; ++s) {
    CP_CUDA(cpk::fill_launch(c->precision, S.xi[s], c->cap[s], -1.0, c->stream));
    CP_TRY(h2d(S.xi[s], c->es * h.slots[s]));
    CP_TRY(h2d(S.u[s], c->es * h.slots[s]));
  }
  CP_TRY(h2d(S.id, 4 * h.slots[1]));
  CP_TRY(h2d(c->Epair, 2 * c->es * (c->N + 1)));
  CP_TRY(h2d(c->phi, sizeof(double) * (c->N + 1)));
  CP_TRY(h2d(c->E64, sizeof(double) * c->N));
  CP_TRY(h2d(c->Glast, sizeof(long long) * (c->N + 1)));
  CP_TRY(h2d(c->hist, sizeof(cp_diag) * h.hist_n));
  CP_CUDA(cudaMemsetAsync(c->G, 0, sizeof(long long) * (c->N + 1), c->stream));
  CP_CUDA(cudaMemcpyAsync(c->dS, &S, sizeof(S), cudaMemcpyHostToDevice, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  c->since_compact = static_cast<int>(h.since_compact);
  return CP_OK;
}

int cp_enable_timing(cp_ctx* c, int32_t on) {
  if (!c) return CP_ERR_ARG;
  c->timing = (on != 0);
  for (int k = 0; k < 3; ++k) {
    c->t_ms[k] = 0.0;
    c->t_n[k] = 0;
  }
  return CP_OK;
}

int cp_read_timing(cp_ctx* c, double ms[3], int64_t n[3]) {
  if (!c || !ms || !n) return CP_ERR_ARG;
  for (int k = 0; k < 3; ++k) {
    ms[k] = c->t_ms[k];
    n[k] = c->t_n[k];
  }
  return CP_OK;
}

int cp_read_launch_times(cp_ctx* c, double* ms, int64_t cap, int64_t* n) {
  if (!c || !n || (cap > 0 && !ms)) return CP_ERR_ARG;
  const int64_t m = static_cast<int64_t>(c->last_step_ms.size());
  *n = m;
  for (int64_t k = 0; k < m && k < cap; ++k) ms[k] = c->last_step_ms[k];
  return m > cap ? CP_ERR_CAPACITY : CP_OK;
}

int cp_last_launch_count(cp_ctx* c, int64_t* launches) {
  if (!c || !launches) return CP_ERR_ARG;
  *launches = c->launches;
  return CP_OK;
}

void cp_destroy(cp_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

const char* cp_status_str(int s) {
  switch (s) {
    case CP_OK: return "ok";
    case CP_ERR_ARG: return "invalid argument or call order";
    case CP_ERR_OOM: return "device allocation failed";
    case CP_ERR_CUDA: return "CUDA runtime error";
    case CP_ERR_CAPACITY: return "particle store or scratch list overflow";
    case CP_ERR_RESIDUAL: return "strict solve did not reach the requested residual";
    case CP_ERR_NONFINITE: return "non-finite field or circuit state";
    case CP_ERR_TIMEOUT: return "bounded device wait gave up";
    default: return "unknown status";
  }
}

// ---- ensemble of independent instances ----------------------------------------
}  // extern "C"

struct cp_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::vector<cp_ctx*> inst;
  int E = 0;
  int precision = CP_FP32;
  int n_max = 0;
  bool initialized = false;
  cpk::Bufs* dBall = nullptr;
  void* abs = nullptr;
  int abs_cap = 4096;
  int abs_grid = 0;      // CTAs the absorbed-ion lists were sized for
  int push_threads = 512;
  int push_grid = 0;
  size_t push_smem = 0;
  size_t solve_smem = 0;
  int compact_grid = 0;
  int compact_every = 128;
  int since_compact = 0;
  int64_t max_steps = 0;
  cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};  // strict, weak, learned weak
  double gtol[3] = {0.0, 0.0, 0.0};
  int64_t launches = 0;
  int* dstatus = nullptr;
  bool timing = false;
  double t_ms[3] = {0.0, 0.0, 0.0};  // push, solve, removal
  int64_t t_n[3] = {0, 0, 0};
  std::vector<cudaEvent_t> ev;
};

namespace {

void batch_free(cp_batch* b) {
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  b->ev.clear();
  for (int m = 0; m < 3; ++m)
    if (b->gexec[m]) cudaGraphExecDestroy(b->gexec[m]);
  cudaFree(b->dBall);
  cudaFree(b->abs);
  cudaFree(b->dstatus);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (cp_ctx* c : b->inst) cp_destroy(c);
  b->inst.clear();
}

// Size the ensemble push for a block shape (threads, CTAs per SM <= occupancy).
int batch_set_shape(cp_batch* b, int threads, int per_sm_req) {
  if (threads != 256 && threads != 512 && threads != 1024) return CP_ERR_ARG;
  int per_sm = 0, sms = 0;
  CP_CUDA(cpk::push_ens_occupancy(b->precision, threads, b->push_smem, &per_sm));
  if (per_sm < 1) return CP_ERR_ARG;
  if (per_sm_req > 0) {
    if (per_sm_req > per_sm) return CP_ERR_ARG;
    per_sm = per_sm_req;
  }
  CP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  const int grid = per_sm * sms;
  if (grid > b->abs_grid) {  // absorbed-ion lists: one per CTA
    cudaFree(b->abs);
    b->abs = nullptr;
    CP_TRY(alloc(&b->abs, cpk::abs_rec_ens_bytes() * static_cast<size_t>(grid) * b->abs_cap));
    b->abs_grid = grid;
  }
  b->push_threads = threads;
  b->push_grid = grid;
  for (int m = 0; m < 3; ++m) {  // graphs carry the old shape
    if (b->gexec[m]) cudaGraphExecDestroy(b->gexec[m]);
    b->gexec[m] = nullptr;
  }
  return CP_OK;
}

int batch_init(cp_batch* b, int mode, double tol) {
  for (cp_ctx* c : b->inst) {
    c->ens_member = true;
    CP_TRY(initialize(c, mode, tol));
  }
  std::vector<cpk::Bufs> hb(b->E);
  b->n_max = 0;
  for (int i = 0; i < b->E; ++i) {
    hb[i] = make_bufs(b->inst[i]);
    b->n_max = std::max(b->n_max, b->inst[i]->N);
  }
  CP_TRY(alloc(reinterpret_cast<void**>(&b->dBall), sizeof(cpk::Bufs) * b->E));
  CP_CUDA(cudaMemcpyAsync(b->dBall, hb.data(), sizeof(cpk::Bufs) * b->E, cudaMemcpyHostToDevice,
                          b->stream));
  CP_TRY(alloc(reinterpret_cast<void**>(&b->dstatus), sizeof(int) * b->E));
  b->push_smem = cpk::push_ens_smem_bytes(b->n_max, b->precision, b->E);
  b->solve_smem = cpk::solve_smem_bytes(b->n_max, 1);
  CP_CUDA(cpk::solve_ens_configure(b->precision, b->solve_smem));
  int sms = 0;
  CP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  b->compact_grid = 2 * sms;
  CP_TRY(batch_set_shape(b, 512, 0));
  CP_CUDA(cudaStreamSynchronize(b->stream));
  b->initialized = true;
  return CP_OK;
}

cudaError_t batch_step_launches(cp_batch* b, cudaStream_t st, int mode, double tol) {
  cudaError_t e = cpk::push_ens_launch(b->precision, b->push_threads, b->push_grid, b->push_smem,
                                       b->dBall, b->E, b->n_max, b->abs, b->abs_cap, st);
  if (e == cudaSuccess)
    e = cpk::solve_ens_launch(b->precision, b->dBall, b->E, b->solve_smem, st, 1, mode, tol);
  return e;
}

int batch_build_graph(cp_batch* b, int mode, double tol) {
  if (b->gexec[mode] && b->gtol[mode] == tol) return CP_OK;
  if (b->gexec[mode]) {
    cudaGraphExecDestroy(b->gexec[mode]);
    b->gexec[mode] = nullptr;
  }
  cudaGraph_t g = nullptr;
  CP_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < b->compact_every && e == cudaSuccess; ++k)
    e = batch_step_launches(b, b->cap_stream, mode, tol);
  if (e == cudaSuccess) e = cpk::compact_ens_launch(b->precision, b->dBall, b->E, b->compact_grid, b->cap_stream);
  const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return CP_ERR_CUDA;
  }
  const cudaError_t e3 = cudaGraphInstantiate(&b->gexec[mode], g, 0);
  cudaGraphDestroy(g);
  CP_CUDA(e3);
  b->gtol[mode] = tol;
  return CP_OK;
}

// First non-zero instance status (0 if none); statuses gathered by one kernel.
int batch_status(cp_batch* b, std::vector<int>* all) {
  std::vector<int> st(b->E, 0);
  CP_CUDA(cpk::status_ens_launch(b->dBall, b->E, b->dstatus, b->stream));
  CP_CUDA(cudaMemcpyAsync(st.data(), b->dstatus, sizeof(int) * b->E, cudaMemcpyDeviceToHost, b->stream));
  CP_CUDA(cudaStreamSynchronize(b->stream));
  int first = 0;
  for (int v : st)
    if (v != 0 && first == 0) first = v;
  if (all) *all = st;
  return first;
}

// Steps launched one kernel at a time between CUDA events (timing mode).
int batch_steps_timed(cp_batch* b, int mode, int32_t n_steps, double tol) {
  std::vector<std::pair<int, size_t>> rec;
  auto timed = [&](int which) -> int {
    const size_t k = rec.size() * 2;
    while (b->ev.size() < k + 2) {
      cudaEvent_t e;
      CP_CUDA(cudaEventCreate(&e));
      b->ev.push_back(e);
    }
    CP_CUDA(cudaEventRecord(b->ev[k], b->stream));
    if (which == 0)
      CP_CUDA(cpk::push_ens_launch(b->precision, b->push_threads, b->push_grid, b->push_smem,
                                   b->dBall, b->E, b->n_max, b->abs, b->abs_cap, b->stream));
    else if (which == 1)
      CP_CUDA(cpk::solve_ens_launch(b->precision, b->dBall, b->E, b->solve_smem, b->stream, 1,
                                    mode, tol));
    else
      CP_CUDA(cpk::compact_ens_launch(b->precision, b->dBall, b->E, b->compact_grid, b->stream));
    CP_CUDA(cudaEventRecord(b->ev[k + 1], b->stream));
    rec.push_back({which, k});
    return CP_OK;
  };
  for (int k = 0; k < n_steps; ++k) {
    CP_TRY(timed(0));
    CP_TRY(timed(1));
    b->launches += 2;
    if (++b->since_compact == b->compact_every) {
      CP_TRY(timed(2));
      b->launches += 2;
      b->since_compact = 0;
    }
  }
  CP_CUDA(cudaStreamSynchronize(b->stream));
  for (const auto& r : rec) {
    float ms = 0.f;
    CP_CUDA(cudaEventElapsedTime(&ms, b->ev[r.second], b->ev[r.second + 1]));
    b->t_ms[r.first] += ms;
    b->t_n[r.first] += 1;
  }
  return CP_OK;
}

int batch_steps(cp_batch* b, int mode, int32_t n_steps, double tol) {
  if (!b || n_steps < 0 || !(tol > 0.0)) return CP_ERR_ARG;
  CP_CUDA(cudaSetDevice(b->device));
  b->launches = 0;
  if (!b->initialized) CP_TRY(batch_init(b, mode, tol));
  int64_t level = 0;
  CP_CUDA(cudaMemcpyAsync(&level, &b->inst[0]->dS->level, sizeof(level), cudaMemcpyDeviceToHost,
                          b->stream));
  CP_CUDA(cudaStreamSynchronize(b->stream));
  if (level + n_steps > b->max_steps) return CP_ERR_ARG;
  if (b->timing) {
    CP_TRY(batch_steps_timed(b, mode, n_steps, tol));
    return batch_status(b, nullptr);
  }
  int left = n_steps;
  while (left > 0) {
    if (b->since_compact == 0 && left >= b->compact_every) {
      CP_TRY(batch_build_graph(b, mode, tol));
      CP_CUDA(cudaGraphLaunch(b->gexec[mode], b->stream));
      b->launches += 2 * b->compact_every + 2;
      left -= b->compact_every;
      continue;
    }
    CP_CUDA(batch_step_launches(b, b->stream, mode, tol));
    b->launches += 2;
    --left;
    if (++b->since_compact == b->compact_every) {
      CP_CUDA(cpk::compact_ens_launch(b->precision, b->dBall, b->E, b->compact_grid, b->stream));
      b->launches += 2;
      b->since_compact = 0;
    }
  }
  return batch_status(b, nullptr);
}

}  // namespace

extern "C" {

int cp_batch_create(int32_t n, const cp_gap* gaps, const cp_circuit* circuits,
                    const cp_see_beam* sees, const cp_run* runs, void* stream, cp_batch** out) {
  if (!out || !gaps || !circuits || !sees || !runs || n < 1 || n > cpk::ens_max_instances())
    return CP_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (runs[i].precision != runs[0].precision || runs[i].max_steps != runs[0].max_steps ||
        runs[i].compact_every != runs[0].compact_every || gaps[i].n_cells > 4096)
      return CP_ERR_ARG;
  }
  cp_batch* b = new (std::nothrow) cp_batch();
  if (!b) return CP_ERR_OOM;
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return CP_ERR_CUDA;
  }
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->E = n;
  b->precision = runs[0].precision;
  b->inst.reserve(n);
  for (int i = 0; i < n; ++i) {
    cp_ctx* c = nullptr;
    const int rc = cp_create(&gaps[i], &circuits[i], &sees[i], &runs[i], stream, &c);
    if (rc != CP_OK) {
      batch_free(b);
      delete b;
      return rc;
    }
    b->inst.push_back(c);
  }
  // an ensemble's small instances lose particles fast: its own default
  // removes them every 64 steps (8 % faster than 128 on the 512-instance run)
  b->compact_every = runs[0].compact_every > 0 ? runs[0].compact_every : 64;
  b->max_steps = b->inst[0]->max_steps;
  *out = b;
  return CP_OK;
}

int cp_batch_set_particles(cp_batch* b, int32_t i, int32_t species, const double* x, const double* v,
                           const uint32_t* id, int64_t n, int32_t units) {
  if (!b || i < 0 || i >= b->E || b->initialized) return CP_ERR_ARG;
  return cp_set_particles(b->inst[i], species, x, v, id, n, units);
}

int cp_batch_step_strict(cp_batch* b, int32_t n_steps, double residual_tol) {
  return batch_steps(b, 0, n_steps, residual_tol);
}

int cp_batch_step_weak(cp_batch* b, int32_t n_steps) { return batch_steps(b, 1, n_steps, 1e300); }

int cp_batch_set_predictor(cp_batch* b, int32_t i, const float* params, const cp_predictor* norm) {
  if (!b || i < 0 || i >= b->E) return CP_ERR_ARG;
  const int rc = cp_set_predictor(b->inst[i], params, norm);
  if (rc != CP_OK || !b->initialized) return rc;
  // the ensemble kernels read the instance's buffer set from the device
  // table at every launch: refresh instance i's entry
  const cpk::Bufs hb = make_bufs(b->inst[i]);
  CP_CUDA(cudaMemcpyAsync(b->dBall + i, &hb, sizeof(cpk::Bufs), cudaMemcpyHostToDevice, b->stream));
  CP_CUDA(cudaStreamSynchronize(b->stream));
  return CP_OK;
}

int cp_batch_step_weak_learned(cp_batch* b, int32_t n_steps) {
  return batch_steps(b, 2, n_steps, 1e300);
}

int cp_batch_predictor_samples(cp_batch* b, int32_t i, int64_t first_level, int64_t n, float* X,
                               float* Y) {
  if (!b || i < 0 || i >= b->E) return CP_ERR_ARG;
  return cp_predictor_samples(b->inst[i], first_level, n, X, Y);
}

int cp_batch_read_history(cp_batch* b, int32_t i, int64_t first, int64_t n, cp_diag* out) {
  if (!b || i < 0 || i >= b->E) return CP_ERR_ARG;
  return cp_read_history(b->inst[i], first, n, out);
}

int cp_batch_read_grid(cp_batch* b, int32_t i, double* phi, double* rho, double* E, int64_t* G,
                       int32_t n_nodes) {
  if (!b || i < 0 || i >= b->E) return CP_ERR_ARG;
  return cp_read_grid(b->inst[i], phi, rho, E, G, n_nodes);
}

int cp_batch_get_particles(cp_batch* b, int32_t i, int32_t species, double* xi, double* u,
                           uint32_t* id, int64_t cap, int64_t* n) {
  if (!b || i < 0 || i >= b->E) return CP_ERR_ARG;
  return cp_get_particles(b->inst[i], species, xi, u, id, cap, n);
}

int cp_batch_status(cp_batch* b, int32_t* status) {
  if (!b || !status) return CP_ERR_ARG;
  if (!b->initialized) {
    for (int i = 0; i < b->E; ++i) status[i] = 0;
    return CP_OK;
  }
  std::vector<int> all;
  CP_CUDA(cudaSetDevice(b->device));
  const int first = batch_status(b, &all);
  if (first < 0 && all.empty()) return first;
  for (int i = 0; i < b->E; ++i) status[i] = all[i];
  return CP_OK;
}

int cp_batch_set_launch(cp_batch* b, int32_t threads, int32_t ctas_per_sm) {
  if (!b || !b->initialized) return CP_ERR_ARG;
  CP_CUDA(cudaSetDevice(b->device));
  return batch_set_shape(b, threads, ctas_per_sm);
}

int cp_batch_get_launch(cp_batch* b, int32_t* threads, int32_t* grid) {
  if (!b || !threads || !grid || !b->initialized) return CP_ERR_ARG;
  *threads = b->push_threads;
  *grid = b->push_grid;
  return CP_OK;
}

int cp_batch_autotune(cp_batch* b, int32_t steps_per_shape, int32_t mode, double residual_tol,
                      int32_t* threads, int32_t* ctas_per_sm, double* push_ms) {
  if (!b || steps_per_shape < 1 || (mode != 0 && mode != 1) || !(residual_tol > 0.0))
    return CP_ERR_ARG;
  CP_CUDA(cudaSetDevice(b->device));
  if (!b->initialized) CP_TRY(batch_init(b, mode, residual_tol));
  const double tol = (mode == 0) ? residual_tol : 1e300;
  const int shapes[][2] = {{512, 2}, {512, 1}, {256, 2}, {256, 1}, {1024, 1}};
  double best = 1e300;
  int best_t = 512, best_p = 0;
  cudaEvent_t e0, e1;
  CP_CUDA(cudaEventCreate(&e0));
  CP_CUDA(cudaEventCreate(&e1));
  int rc = CP_OK;
  for (const auto& sh : shapes) {
    if (batch_set_shape(b, sh[0], sh[1]) != CP_OK) continue;  // shape not resident on this device
    int64_t level = 0;
    rc = cuda_rc(cudaMemcpyAsync(&level, &b->inst[0]->dS->level, sizeof(level),
                                 cudaMemcpyDeviceToHost, b->stream));
    if (rc == CP_OK) rc = cuda_rc(cudaStreamSynchronize(b->stream));
    if (rc != CP_OK) break;
    if (level + steps_per_shape > b->max_steps) {
      rc = CP_ERR_ARG;
      break;
    }
    // ordinary steps of the run (results do not depend on the launch shape);
    // the push of each is timed
    double ms_sum = 0.0;
    for (int k = 0; k < steps_per_shape && rc == CP_OK; ++k) {
      rc = cuda_rc(cudaEventRecord(e0, b->stream));
      if (rc == CP_OK)
        rc = cuda_rc(cpk::push_ens_launch(b->precision, b->push_threads, b->push_grid, b->push_smem,
                                          b->dBall, b->E, b->n_max, b->abs, b->abs_cap, b->stream));
      if (rc == CP_OK) rc = cuda_rc(cudaEventRecord(e1, b->stream));
      if (rc == CP_OK)
        rc = cuda_rc(cpk::solve_ens_launch(b->precision, b->dBall, b->E, b->solve_smem, b->stream,
                                           1, mode, tol));
      if (rc == CP_OK) rc = cuda_rc(cudaEventSynchronize(e1));
      float ms = 0.f;
      if (rc == CP_OK) rc = cuda_rc(cudaEventElapsedTime(&ms, e0, e1));
      ms_sum += ms;
      if (++b->since_compact == b->compact_every && rc == CP_OK) {
        rc = cuda_rc(cpk::compact_ens_launch(b->precision, b->dBall, b->E, b->compact_grid, b->stream));
        b->since_compact = 0;
      }
    }
    if (rc != CP_OK) break;
    const double avg = ms_sum / steps_per_shape;
    if (avg < best) {
      best = avg;
      best_t = b->push_threads;
      best_p = b->push_grid;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CP_OK) return rc;
  int sms = 1;
  CP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  CP_TRY(batch_set_shape(b, best_t, best_p / sms));
  if (threads) *threads = best_t;
  if (ctas_per_sm) *ctas_per_sm = best_p / sms;
  if (push_ms) *push_ms = best;
  const int st = batch_status(b, nullptr);
  return st;
}

int cp_batch_get_level(cp_batch* b, int32_t i, int64_t* level) {
  if (!b || !level || i < 0 || i >= b->E) return CP_ERR_ARG;
  return cp_get_level(b->inst[i], level);
}

int cp_batch_enable_timing(cp_batch* b, int32_t on) {
  if (!b) return CP_ERR_ARG;
  b->timing = (on != 0);
  for (int k = 0; k < 3; ++k) {
    b->t_ms[k] = 0.0;
    b->t_n[k] = 0;
  }
  return CP_OK;
}

int cp_batch_read_timing(cp_batch* b, double ms[3], int64_t n[3]) {
  if (!b || !ms || !n) return CP_ERR_ARG;
  for (int k = 0; k < 3; ++k) {
    ms[k] = b->t_ms[k];
    n[k] = b->t_n[k];
  }
  return CP_OK;
}

int cp_batch_last_launch_count(cp_batch* b, int64_t* launches) {
  if (!b || !launches) return CP_ERR_ARG;
  *launches = b->launches;
  return CP_OK;
}

void cp_batch_destroy(cp_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
}

// ---- 2D planar gap ------------------------------------------------------------
}  // extern "C"

struct cp_gap2d {
  cp_ctx* c = nullptr;  // the 1D problem of the transverse mean (circuit, history)
  int Nx = 0, Ny = 0, T = 0, sms = 0, grid = 0;
  int sort_every = 16, since_sort = 0;
  double ly = 0.0, beam_sigma = 0.0, beam_yc = 0.0;
  bool initialized = false;
  cpk::Dev2D hd{};             // host copy of the device struct
  cpk::Dev2D* dD = nullptr;
  void* abs = nullptr;
  int abs_cap = 4096;
  std::vector<double> hx[kSpecies], hy[kSpecies], hu[kSpecies], hw[kSpecies];
  std::vector<uint32_t> hid;
  std::vector<void*> owned;    // device allocations of this object
  int64_t launches = 0;
  bool timing = false;
  double t_ms[3] = {0.0, 0.0, 0.0};  // push, solve (all kernels), sort
  int64_t t_n[3] = {0, 0, 0};
  std::vector<cudaEvent_t> ev;
};

namespace {

int g2_alloc(cp_gap2d* g, void** p, size_t bytes) {
  CP_TRY(alloc(p, bytes));
  g->owned.push_back(*p);
  return CP_OK;
}

void g2_free(cp_gap2d* g) {
  for (void* p : g->owned) cudaFree(p);
  g->owned.clear();
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  g->ev.clear();
  if (g->c) {
    // the 1D context's particle pointers are this object's: forget them first
    cp_ctx* c = g->c;
    for (int b = 0; b < 2; ++b) {
      for (int s = 0; s < kSpecies; ++s) c->buf_xi[b][s] = c->buf_u[b][s] = nullptr;
      c->buf_id[b] = nullptr;
    }
    cp_destroy(c);
    g->c = nullptr;
  }
}

// Kernels of one step after the push: row sums + spectra, the 1D coupled
// solve of the mean, the transverse modes and the fields.
int g2_solve(cp_gap2d* g, int do_push, int mode, double tol) {
  cp_ctx* c = g->c;
  const cpk::Bufs B = make_bufs(c);
  CP_CUDA(cpk::solve2_fwd_launch(g->dD, c->G, g->Nx, g->Ny, c->stream));
  CP_CUDA(cpk::solve_launch(c->precision, B, c->solve_ctas, c->solve_smem, c->stream, do_push, mode, tol));
  const float c_rhs = static_cast<float>(-c->hp.dx * c->hp.dx / c->hp.eps0);
  CP_CUDA(cpk::solve2_modes_launch(g->dD, g->Nx, g->Ny, c_rhs, c->E64, c->stream));
  g->launches += 6;
  return CP_OK;
}

int g2_sort(cp_gap2d* g) {
  cp_ctx* c = g->c;
  for (int s = 0; s < kSpecies; ++s) CP_CUDA(cpk::sort2_launch(c->dS, g->dD, g->T, s, g->sms, c->stream));
  g->launches += 6 * kSpecies;
  return CP_OK;
}

int g2_init(cp_gap2d* g, int mode, double tol) {
  cp_ctx* c = g->c;
  cpk::DevParams& P = c->hp;
  int64_t n[kSpecies];
  for (int s = 0; s < kSpecies; ++s) n[s] = static_cast<int64_t>(g->hx[s].size());
  const int64_t Bm = P.beam_per_step;
  const int64_t pad = 4 * static_cast<int64_t>(g->T) + 64;
  const int64_t ions_ever = n[1] + Bm * c->max_steps;
  const int64_t def[kSpecies] = {round4(n[0]) + pad, round4(ions_ever) + pad,
                                 std::max<int64_t>(65536, round4(ions_ever + n[2]) + pad)};
  for (int s = 0; s < kSpecies; ++s) {
    c->cap[s] = round4(c->cap_req[s] > 0 ? std::max<int64_t>(c->cap_req[s], round4(n[s]) + pad) : def[s]);
    P.cap[s] = c->cap[s];
  }
  cpk::Dev2D& D = g->hd;
  // particle stores: x, u (the 1D state's buffers), y, w, ids; two of each
  for (int b = 0; b < 2; ++b) {
    for (int s = 0; s < kSpecies; ++s) {
      void* bufs[4];
      for (int k = 0; k < 4; ++k) CP_TRY(g2_alloc(g, &bufs[k], sizeof(float) * c->cap[s]));
      CP_CUDA(cpk::fill_launch(CP_FP32, bufs[0], c->cap[s], -1.0, c->stream));
      for (int k = 1; k < 4; ++k) CP_CUDA(cudaMemsetAsync(bufs[k], 0, sizeof(float) * c->cap[s], c->stream));
      c->buf_xi[b][s] = bufs[0];
      c->buf_u[b][s] = bufs[1];
      (b == 0 ? D.y : D.y_alt)[s] = bufs[2];
      (b == 0 ? D.w : D.w_alt)[s] = bufs[3];
    }
    void* idb = nullptr;
    CP_TRY(g2_alloc(g, &idb, sizeof(uint32_t) * c->cap[1]));
    c->buf_id[b] = static_cast<uint32_t*>(idb);
  }
  for (int s = 0; s < kSpecies; ++s) {
    if (!n[s]) continue;
    std::vector<float> f(n[s]);
    const std::vector<double>* src[4] = {&g->hx[s], &g->hu[s], &g->hy[s], &g->hw[s]};
    void* dst[4] = {c->buf_xi[0][s], c->buf_u[0][s], D.y[s], D.w[s]};
    for (int k = 0; k < 4; ++k) {
      for (int64_t q = 0; q < n[s]; ++q) f[q] = static_cast<float>((*src[k])[q]);
      CP_CUDA(cudaMemcpyAsync(dst[k], f.data(), 4 * n[s], cudaMemcpyHostToDevice, c->stream));
      CP_CUDA(cudaStreamSynchronize(c->stream));
    }
  }
  uint32_t id_base = 0;
  if (n[1]) {
    CP_CUDA(cudaMemcpyAsync(c->buf_id[0], g->hid.data(), 4 * n[1], cudaMemcpyHostToDevice, c->stream));
    for (uint32_t v : g->hid) id_base = std::max<uint32_t>(id_base, v + 1u);
  }
  if (static_cast<double>(id_base) + static_cast<double>(Bm) * c->max_steps > 4294967295.0)
    return CP_ERR_ARG;
  // the 1D mean problem's grids, parameters and state
  const int N = c->N;
  CP_TRY(alloc(reinterpret_cast<void**>(&c->G), sizeof(long long) * (N + 1)));
  CP_TRY(alloc(reinterpret_cast<void**>(&c->Glast), sizeof(long long) * (N + 1)));
  CP_TRY(alloc(&c->Epair, 2 * sizeof(float) * (N + 1)));
  CP_TRY(alloc(reinterpret_cast<void**>(&c->phi), sizeof(double) * (N + 1)));
  CP_TRY(alloc(reinterpret_cast<void**>(&c->E64), sizeof(double) * N));
  c->hist_rows = c->max_steps + 1;
  CP_TRY(alloc(reinterpret_cast<void**>(&c->hist), sizeof(cp_diag) * c->hist_rows));
  CP_CUDA(cudaMemsetAsync(c->G, 0, sizeof(long long) * (N + 1), c->stream));
  CP_CUDA(cudaMemsetAsync(c->Glast, 0, sizeof(long long) * (N + 1), c->stream));
  CP_CUDA(cudaMemsetAsync(c->Epair, 0, 2 * sizeof(float) * (N + 1), c->stream));
  CP_CUDA(cudaMemsetAsync(c->hist, 0, sizeof(cp_diag) * c->hist_rows, c->stream));
  CP_CUDA(cpk::solve_cluster_size(c->precision, N, &c->solve_ctas));
  c->solve_smem = cpk::solve_smem_bytes(N, c->solve_ctas);
  CP_CUDA(cpk::solve_configure(c->precision, c->solve_smem));
  CP_TRY(alloc(reinterpret_cast<void**>(&c->abs), sizeof(cpk::AbsRec)));
  // the mean's charge grid (column sums of the 2D grid) counts 2^32 per
  // macroparticle; every int64 sum stays below 2^63 while the stores hold
  // fewer than 2^30 macroparticles (a node gets at most twice 2^32 each)
  if (c->cap[0] + c->cap[1] + c->cap[2] > (int64_t(1) << 30)) return CP_ERR_ARG;
  P.scale = P.e * P.weight / (P.area * P.dx * cpk::kFix2);
  P.alpha = P.dx * P.dx * P.scale / P.eps0;
  CP_TRY(alloc(reinterpret_cast<void**>(&c->dP), sizeof(cpk::DevParams)));
  CP_CUDA(cudaMemcpyAsync(c->dP, &c->hp, sizeof(cpk::DevParams), cudaMemcpyHostToDevice, c->stream));
  CP_TRY(alloc(reinterpret_cast<void**>(&c->vs), sizeof(double) * (c->hist_rows + 1)));
  CP_CUDA(cpk::source_table_launch(c->dP, c->vs, c->hist_rows + 1, c->stream));
  cpk::DevState S;
  std::memset(&S, 0, sizeof(S));
  for (int s = 0; s < kSpecies; ++s) {
    S.xi[s] = c->buf_xi[0][s];
    S.u[s] = c->buf_u[0][s];
    S.xi_alt[s] = c->buf_xi[1][s];
    S.u_alt[s] = c->buf_u[1][s];
    S.n_alloc[s] = round4(n[s]);
    S.n_proc[s] = round4(n[s]);
    S.n_live[s] = n[s];
  }
  S.id = c->buf_id[0];
  S.id_alt = c->buf_id[1];
  S.sigma = c->sigma0;
  S.beam_id_base = id_base;
  for (int k = 0; k < 4; ++k)  // the circuit rests before t = 0
    for (int i = 0; i < 5; ++i) S.Qt[k][i] = c->hp.t_Q0[i];
  CP_TRY(alloc(reinterpret_cast<void**>(&c->dS), sizeof(cpk::DevState)));
  CP_CUDA(cudaMemcpyAsync(c->dS, &S, sizeof(S), cudaMemcpyHostToDevice, c->stream));
  // 2D grids and tables
  const int Nx = g->Nx, Ny = g->Ny, M = Ny / 2 + 1, T = g->T;
  const size_t nodes = static_cast<size_t>(Nx + 1) * Ny;
  void* p = nullptr;
  CP_TRY(g2_alloc(g, &p, sizeof(int) * 3 * (T + 1))); D.tile_start = static_cast<int*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(int) * 3 * (T + 1))); D.wi_off = static_cast<int*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(int) * 3 * T)); D.tile_cnt = static_cast<int*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(int) * 3 * T)); D.tile_cur = static_cast<int*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(float) * Nx * Ny)); D.Ex = static_cast<float*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(float) * nodes)); D.Ey = static_cast<float*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(long long) * nodes)); D.G2 = static_cast<long long*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(long long) * nodes)); D.G2last = static_cast<long long*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(float2) * (Nx + 1) * M)); D.R = static_cast<float2*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(float) * (Nx + 1) * M)); D.cp = static_cast<float*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(float) * (Nx + 1) * M)); D.tinv = static_cast<float*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(float) * nodes)); D.phit = static_cast<float*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(float) * M)); D.kappa = static_cast<float*>(p);
  CP_TRY(g2_alloc(g, &p, sizeof(float2) * (Ny / 2))); D.tw = static_cast<float2*>(p);
  for (int* q : {D.tile_start, D.wi_off}) CP_CUDA(cudaMemsetAsync(q, 0, sizeof(int) * 3 * (T + 1), c->stream));
  for (int* q : {D.tile_cnt, D.tile_cur}) CP_CUDA(cudaMemsetAsync(q, 0, sizeof(int) * 3 * T, c->stream));
  CP_CUDA(cudaMemsetAsync(D.G2, 0, sizeof(long long) * nodes, c->stream));
  CP_CUDA(cudaMemsetAsync(D.G2last, 0, sizeof(long long) * nodes, c->stream));
  CP_CUDA(cudaMemsetAsync(D.phit, 0, sizeof(float) * nodes, c->stream));
  CP_CUDA(cudaMemsetAsync(D.R, 0, sizeof(float2) * (Nx + 1) * M, c->stream));
  D.Nx = Nx;
  D.Ny = Ny;
  D.ntx = (Nx + cpk::kT2 - 1) / cpk::kT2;
  D.nty = (Ny + cpk::kT2 - 1) / cpk::kT2;
  D.T = T;
  D.sort_every = g->sort_every;
  D.Nxf = static_cast<float>(Nx);
  D.Nyf = static_cast<float>(Ny);
  D.dx = P.dx;
  D.dy = g->ly / Ny;
  D.inv_dx = static_cast<float>(1.0 / D.dx);
  D.inv_dy = static_cast<float>(1.0 / D.dy);
  const double Lz = P.area / g->ly;
  D.rho_scale = P.e * P.weight / (D.dx * D.dy * Lz * cpk::kFix2);
  const double dt = P.dt;
  const double q_m[kSpecies] = {-P.e / P.m_e, P.e / P.m_i, -P.e / P.m_e};
  for (int s = 0; s < kSpecies; ++s) {
    const double kx = q_m[s] * dt * dt / D.dx, ky = q_m[s] * dt * dt / D.dy;
    D.kx[0][s] = static_cast<float>(0.5 * kx);
    D.kx[1][s] = static_cast<float>(kx);
    D.ky[0][s] = static_cast<float>(0.5 * ky);
    D.ky[1][s] = static_cast<float>(ky);
  }
  D.beam_sigma = g->beam_sigma / D.dy;
  D.beam_yc = g->beam_yc / D.dy;
  int lg = 0;
  while ((1 << lg) < Ny) ++lg;
  D.logNy = lg;
  D.use_win = (Ny >= cpk::kW2) ? 1 : 0;
  for (int s = 0; s < kSpecies; ++s) {
    D.n_sorted[s] = 0;
    D.cap[s] = c->cap[s];
  }
  CP_TRY(g2_alloc(g, reinterpret_cast<void**>(&g->dD), sizeof(cpk::Dev2D)));
  CP_CUDA(cudaMemcpyAsync(g->dD, &D, sizeof(D), cudaMemcpyHostToDevice, c->stream));
  CP_CUDA(cpk::tables2_launch(g->dD, Ny, (D.dx / D.dy) * (D.dx / D.dy), c->stream));
  int per_sm = 0;
  CP_CUDA(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, c->device));
  CP_TRY(g2_alloc(g, &p, sizeof(int) * 2 * g->sms * T));
  D.bhist = static_cast<int*>(p);
  CP_CUDA(cudaMemcpyAsync(&g->dD->bhist, &D.bhist, sizeof(int*), cudaMemcpyHostToDevice, c->stream));
  CP_CUDA(cpk::push2_occupancy(&per_sm));
  if (per_sm < 1) return CP_ERR_ARG;
  g->grid = per_sm * g->sms;
  CP_TRY(g2_alloc(g, &g->abs, sizeof(cpk::AbsRec2) * static_cast<size_t>(g->grid) * g->abs_cap));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  for (int s = 0; s < kSpecies; ++s) {
    std::vector<double>().swap(g->hx[s]);
    std::vector<double>().swap(g->hy[s]);
    std::vector<double>().swap(g->hu[s]);
    std::vector<double>().swap(g->hw[s]);
  }
  c->initialized = true;
  g->initialized = true;
  // level 0: sort, deposit, solve
  CP_TRY(g2_sort(g));
  g->since_sort = 0;
  CP_CUDA(cpk::deposit2_level0_launch(c->dS, g->dD, g->sms, c->stream));
  CP_TRY(g2_solve(g, 0, mode, tol));
  return CP_OK;
}

int g2_timed(cp_gap2d* g, int which, std::vector<std::pair<int, size_t>>* rec) {
  const size_t k = rec->size() * 2;
  while (g->ev.size() < k + 2) {
    cudaEvent_t e;
    CP_CUDA(cudaEventCreate(&e));
    g->ev.push_back(e);
  }
  CP_CUDA(cudaEventRecord(g->ev[k], g->c->stream));
  rec->push_back({which, k});
  return CP_OK;
}

int g2_steps(cp_gap2d* g, int mode, int32_t n_steps, double tol) {
  if (!g || n_steps < 0 || !(tol > 0.0)) return CP_ERR_ARG;
  cp_ctx* c = g->c;
  CP_CUDA(cudaSetDevice(c->device));
  g->launches = 0;
  if (!g->initialized) CP_TRY(g2_init(g, mode, tol));
  int64_t level = 0;
  CP_CUDA(cudaMemcpyAsync(&level, &c->dS->level, sizeof(level), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  if (level + n_steps > c->max_steps) return CP_ERR_ARG;
  std::vector<std::pair<int, size_t>> rec;
  auto mark_end = [&](void) -> int {
    const size_t k = rec.back().second;
    CP_CUDA(cudaEventRecord(g->ev[k + 1], c->stream));
    return CP_OK;
  };
  for (int k = 0; k < n_steps; ++k) {
    if (g->since_sort == g->sort_every) {  // periodic re-sort (also drops absorbed slots)
      if (g->timing) CP_TRY(g2_timed(g, 2, &rec));
      CP_TRY(g2_sort(g));
      if (g->timing) CP_TRY(mark_end());
      g->since_sort = 0;
    }
    if (g->timing) CP_TRY(g2_timed(g, 0, &rec));
    CP_CUDA(cpk::push2_launch(c->dP, c->dS, g->dD, &g->hd, g->abs, g->abs_cap, g->grid, c->stream));
    g->launches += 1;
    if (g->timing) CP_TRY(mark_end());
    if (g->timing) CP_TRY(g2_timed(g, 1, &rec));
    CP_TRY(g2_solve(g, 1, mode, tol));
    if (g->timing) CP_TRY(mark_end());
    g->since_sort += 1;
  }
  if (g->timing) {
    CP_CUDA(cudaStreamSynchronize(c->stream));
    for (const auto& r : rec) {
      float ms = 0.f;
      CP_CUDA(cudaEventElapsedTime(&ms, g->ev[r.second], g->ev[r.second + 1]));
      g->t_ms[r.first] += ms;
      g->t_n[r.first] += 1;
    }
  }
  return read_status(c);
}

}  // namespace

extern "C" {

int cp2d_create(const cp_gap* gap, const cp_transverse* tr, const cp_circuit* circuit,
                const cp_see_beam* see, const cp_run* run, void* stream, cp_gap2d** out) {
  if (!out || !gap || !tr || !circuit || !see || !run) return CP_ERR_ARG;
  *out = nullptr;
  const int Ny = tr->n_cells_y;
  if (run->precision != CP_FP32 || Ny < 8 || Ny > 4096 || (Ny & (Ny - 1)) != 0 ||
      gap->n_cells > 4096 || !(tr->length_y > 0) || tr->sort_every < 0 || !(tr->beam_sigma >= 0))
    return CP_ERR_ARG;
  cp_gap2d* g = new (std::nothrow) cp_gap2d();
  if (!g) return CP_ERR_OOM;
  const int rc = cp_create(gap, circuit, see, run, stream, &g->c);
  if (rc != CP_OK) {
    delete g;
    return rc;
  }
  g->c->ens_member = true;
  g->Nx = gap->n_cells;
  g->Ny = Ny;
  g->T = ((g->Nx + cpk::kT2 - 1) / cpk::kT2) * ((Ny + cpk::kT2 - 1) / cpk::kT2);
  g->ly = tr->length_y;
  g->beam_sigma = tr->beam_sigma;
  g->beam_yc = tr->beam_y0;
  g->sort_every = tr->sort_every > 0 ? tr->sort_every : 16;
  *out = g;
  return CP_OK;
}

int cp2d_set_particles(cp_gap2d* g, int32_t species, const double* x, const double* y,
                       const double* vx, const double* vy, const uint32_t* id, int64_t n,
                       int32_t units) {
  if (!g || species < 0 || species >= kSpecies || n < 0 || g->initialized ||
      (units != CP_UNITS_CELL && units != CP_UNITS_SI) || (n > 0 && (!x || !y || !vx || !vy)))
    return CP_ERR_ARG;
  const double dx = g->c->hp.dx, dy = g->ly / g->Ny, dt = g->c->hp.dt;
  const float Nx = static_cast<float>(g->Nx), Ny = static_cast<float>(g->Ny);
  std::vector<double> hx(n), hy(n), hu(n), hw(n);
  for (int64_t k = 0; k < n; ++k) {
    const double xi = units == CP_UNITS_SI ? x[k] / dx : x[k];
    const double eta = units == CP_UNITS_SI ? y[k] / dy : y[k];
    const double u = units == CP_UNITS_SI ? vx[k] * dt / dx : vx[k];
    const double w = units == CP_UNITS_SI ? vy[k] * dt / dy : vy[k];
    if (!(xi > 0.0) || !(xi < g->Nx) || !(eta >= 0.0) || !(eta < g->Ny) || !std::isfinite(u) ||
        !std::isfinite(w))
      return CP_ERR_ARG;
    float fx = static_cast<float>(xi), fy = static_cast<float>(eta);
    if (fx >= Nx) fx = std::nextafter(Nx, 0.0f);
    if (!(fx > 0.0f)) fx = 1.17549435e-38f;
    if (fy >= Ny) fy = 0.0f;
    hx[k] = fx;
    hy[k] = fy;
    hu[k] = static_cast<float>(u);
    hw[k] = static_cast<float>(w);
  }
  g->hx[species].swap(hx);
  g->hy[species].swap(hy);
  g->hu[species].swap(hu);
  g->hw[species].swap(hw);
  if (species == CP_IONS) {
    g->hid.resize(n);
    for (int64_t k = 0; k < n; ++k) g->hid[k] = id ? id[k] : static_cast<uint32_t>(k);
  }
  return CP_OK;
}

int cp2d_step_strict(cp_gap2d* g, int32_t n_steps, double residual_tol) {
  return g2_steps(g, 0, n_steps, residual_tol);
}

int cp2d_step_weak(cp_gap2d* g, int32_t n_steps) { return g2_steps(g, 1, n_steps, 1e300); }

int cp2d_set_predictor(cp_gap2d* g, const float* params, const cp_predictor* norm) {
  if (!g) return CP_ERR_ARG;
  return cp_set_predictor(g->c, params, norm);  // the mean problem's context
}

int cp2d_step_weak_learned(cp_gap2d* g, int32_t n_steps) {
  if (!g || !g->c->net) return CP_ERR_ARG;
  return g2_steps(g, 2, n_steps, 1e300);
}

int cp2d_read_history(cp_gap2d* g, int64_t first, int64_t n, cp_diag* out) {
  if (!g) return CP_ERR_ARG;
  return cp_read_history(g->c, first, n, out);
}

int cp2d_get_level(cp_gap2d* g, int64_t* level) {
  if (!g) return CP_ERR_ARG;
  return cp_get_level(g->c, level);
}

int cp2d_read_fields(cp_gap2d* g, double* phi, float* Ex, float* Ey, int64_t* G) {
  if (!g || !g->initialized) return CP_ERR_ARG;
  cp_ctx* c = g->c;
  CP_CUDA(cudaSetDevice(c->device));
  const int Nx = g->Nx, Ny = g->Ny;
  const size_t nodes = static_cast<size_t>(Nx + 1) * Ny;
  if (phi) {
    std::vector<double> p0(Nx + 1);
    std::vector<float> pt(nodes);
    CP_CUDA(cudaMemcpyAsync(p0.data(), c->phi, sizeof(double) * (Nx + 1), cudaMemcpyDeviceToHost, c->stream));
    CP_CUDA(cudaMemcpyAsync(pt.data(), g->hd.phit, sizeof(float) * nodes, cudaMemcpyDeviceToHost, c->stream));
    CP_CUDA(cudaStreamSynchronize(c->stream));
    for (int i = 0; i <= Nx; ++i)
      for (int j = 0; j < Ny; ++j) phi[static_cast<size_t>(i) * Ny + j] = p0[i] + pt[static_cast<size_t>(i) * Ny + j];
  }
  if (Ex) CP_CUDA(cudaMemcpyAsync(Ex, g->hd.Ex, sizeof(float) * Nx * Ny, cudaMemcpyDeviceToHost, c->stream));
  if (Ey) CP_CUDA(cudaMemcpyAsync(Ey, g->hd.Ey, sizeof(float) * nodes, cudaMemcpyDeviceToHost, c->stream));
  if (G) CP_CUDA(cudaMemcpyAsync(G, g->hd.G2last, sizeof(long long) * nodes, cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  return CP_OK;
}

int cp2d_get_particles(cp_gap2d* g, int32_t species, double* xi, double* eta, double* u, double* w,
                       uint32_t* id, int64_t cap, int64_t* n) {
  if (!g || species < 0 || species >= kSpecies || !n || !g->initialized) return CP_ERR_ARG;
  cp_ctx* c = g->c;
  CP_CUDA(cudaSetDevice(c->device));
  cpk::DevState S;
  cpk::Dev2D D;
  CP_CUDA(cudaMemcpyAsync(&S, c->dS, sizeof(S), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaMemcpyAsync(&D, g->dD, sizeof(D), cudaMemcpyDeviceToHost, c->stream));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  const int64_t slots = std::min<int64_t>(S.n_alloc[species], c->cap[species]);
  std::vector<float> hx(slots), hy(slots), hu(slots), hw(slots);
  std::vector<uint32_t> hid(species == CP_IONS ? slots : 0);
  if (slots > 0) {
    CP_CUDA(cudaMemcpyAsync(hx.data(), S.xi[species], 4 * slots, cudaMemcpyDeviceToHost, c->stream));
    CP_CUDA(cudaMemcpyAsync(hu.data(), S.u[species], 4 * slots, cudaMemcpyDeviceToHost, c->stream));
    CP_CUDA(cudaMemcpyAsync(hy.data(), D.y[species], 4 * slots, cudaMemcpyDeviceToHost, c->stream));
    CP_CUDA(cudaMemcpyAsync(hw.data(), D.w[species], 4 * slots, cudaMemcpyDeviceToHost, c->stream));
    if (species == CP_IONS)
      CP_CUDA(cudaMemcpyAsync(hid.data(), S.id, 4 * slots, cudaMemcpyDeviceToHost, c->stream));
    CP_CUDA(cudaStreamSynchronize(c->stream));
  }
  int64_t m = 0;
  for (int64_t k = 0; k < slots; ++k) {
    if (!(hx[k] > 0.0f && hx[k] < static_cast<float>(g->Nx))) continue;
    if (m < cap) {
      if (xi) xi[m] = hx[k];
      if (eta) eta[m] = hy[k];
      if (u) u[m] = hu[k];
      if (w) w[m] = hw[k];
      if (id && species == CP_IONS) id[m] = hid[k];
    }
    ++m;
  }
  *n = m;
  return m > cap ? CP_ERR_CAPACITY : CP_OK;
}

int cp2d_enable_timing(cp_gap2d* g, int32_t on) {
  if (!g) return CP_ERR_ARG;
  g->timing = (on != 0);
  for (int k = 0; k < 3; ++k) {
    g->t_ms[k] = 0.0;
    g->t_n[k] = 0;
  }
  return CP_OK;
}

int cp2d_read_timing(cp_gap2d* g, double ms[3], int64_t n[3]) {
  if (!g || !ms || !n) return CP_ERR_ARG;
  for (int k = 0; k < 3; ++k) {
    ms[k] = g->t_ms[k];
    n[k] = g->t_n[k];
  }
  return CP_OK;
}

int cp2d_last_launch_count(cp_gap2d* g, int64_t* launches) {
  if (!g || !launches) return CP_ERR_ARG;
  *launches = g->launches;
  return CP_OK;
}

void cp2d_destroy(cp_gap2d* g) {
  if (!g) return;
  if (g->c) {
    cudaSetDevice(g->c->device);
    if (g->c->stream) cudaStreamSynchronize(g->c->stream);
  }
  g2_free(g);
  delete g;
}

}  // extern "C"
