// cp_solve.cu -- the coupled field/circuit solve of a new time level.
//
// k_solve (one thread-block cluster of 8 or 16 CTAs x 512 threads) solves the
//   level: the bordered tridiagonal system of App. B with the circuit row of
//   Sec. 2.4.2 (strict, Eq. Poisson_BC2) or Sec. 2.4.3 (weak, Eq.
//   Poisson_BC3) is factorised into two bidiagonal scans whose charge sums
//   are exact integers (one associative segment scan gives the int64 prefix
//   of the charge grid and the int128 prefix of that); FP64 enters only at
//   the final scaling, so the solve is direct and its backward error is
//   checked over every row and the circuit row, with FP64 iterative
//   refinement if it exceeds the requested tolerance.  Chunk totals are
//   exchanged through distributed shared memory.
#include "cp_common.cuh"
#include "cp_mlp.cuh"

namespace cpk {
// ---------------------------------------------------------------------------
// Scans and reductions for the cluster solve
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long shfl_up_t(long long v, int o) {
  return __shfl_up_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ double shfl_up_t(double v, int o) {
  return __shfl_up_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ __int128 shfl_up_t(__int128 v, int o) {
  const unsigned long long lo = static_cast<unsigned long long>(v);
  const unsigned long long hi = static_cast<unsigned long long>(static_cast<unsigned __int128>(v) >> 64);
  const unsigned long long l2 = __shfl_up_sync(0xffffffffu, lo, o);
  const unsigned long long h2 = __shfl_up_sync(0xffffffffu, hi, o);
  return static_cast<__int128>((static_cast<unsigned __int128>(h2) << 64) | l2);
}

// Sign-magnitude conversion: both 64-bit halves of |v| are non-negative, so
// hi 2^64 + lo has no cancellation (error below 1 ulp of |v|).
__device__ __forceinline__ double i128_to_double(__int128 v) {
  const bool neg = v < 0;
  const unsigned __int128 m = neg ? static_cast<unsigned __int128>(-v) : static_cast<unsigned __int128>(v);
  const unsigned long long hi = static_cast<unsigned long long>(m >> 64);
  const unsigned long long lo = static_cast<unsigned long long>(m);
  const double d = fma(static_cast<double>(hi), 18446744073709551616.0, static_cast<double>(lo));
  return neg ? -d : d;
}

// In-place inclusive scan of a[idx(m)], m = 0..n-1 (idx = m, or n-1-m for a
// suffix scan), contiguous runs per thread; returns the CTA total.
template <typename T>
__device__ T cta_scan(T* a, int n, bool reverse, T* wsum) {
  const int per = (n + kSolveThreads - 1) / kSolveThreads;
  const int lo = min(static_cast<int>(threadIdx.x) * per, n);
  const int hi = min(lo + per, n);
  T s = T(0);
  for (int m = lo; m < hi; ++m) s += a[reverse ? n - 1 - m : m];
  T incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = shfl_up_t(incl, o);
    if (static_cast<int>(lane_id()) >= o) incl += y;
  }
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 31) wsum[w] = incl;
  __syncthreads();
  if (threadIdx.x < 32) {
    T t = (threadIdx.x < kSolveThreads / 32) ? wsum[threadIdx.x] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = shfl_up_t(t, o);
      if (static_cast<int>(threadIdx.x) >= o) t += y;
    }
    wsum[threadIdx.x] = t;
  }
  __syncthreads();
  T run = (w > 0 ? wsum[w - 1] : T(0)) + (incl - s);
  for (int m = lo; m < hi; ++m) {
    const int k = reverse ? n - 1 - m : m;
    run += a[k];
    a[k] = run;
  }
  const T total = wsum[kSolveThreads / 32 - 1];
  __syncthreads();
  return total;
}

__device__ double cta_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < kSolveThreads / 32; ++k) t = fmax(t, red[k]);
  __syncthreads();
  return t;
}

__device__ double cta_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < kSolveThreads / 32; ++k) t += red[k];
  __syncthreads();
  return t;
}

// Exclusive prefix (in rank order, or reverse rank order) and total over the
// cluster of one value per CTA, through distributed shared memory.
template <typename T>
__device__ void cluster_prefix(T mine, T* slot, bool reverse, T* excl, T* total) {
  cg::cluster_group cl = cg::this_cluster();
  if (threadIdx.x == 0) *slot = mine;
  cl.sync();
  const unsigned me = cl.block_rank();
  const unsigned nr = cl.num_blocks();
  T acc = T(0), tot = T(0);
  for (unsigned r = 0; r < nr; ++r) {
    const T v = *cl.map_shared_rank(slot, r);
    if (reverse ? (r > me) : (r < me)) acc += v;
    tot += v;
  }
  *excl = acc;
  *total = tot;
  cl.sync();
}

__device__ double cluster_max(double mine, double* slot) {
  cg::cluster_group cl = cg::this_cluster();
  if (threadIdx.x == 0) *slot = mine;
  cl.sync();
  double m = 0.0;
  for (unsigned r = 0; r < cl.num_blocks(); ++r) m = fmax(m, *cl.map_shared_rank(slot, r));
  cl.sync();
  return m;
}

// FP64 direct solve of the same tridiagonal system for an arbitrary right-hand
// side (used by the refinement sweeps): on entry v[k] = b_{lo+k}, b0 = b_0;
// on exit v[k] = x_{lo+k}.  D_i = D_0 - sum_{j=1..i} b_j, D_0 = b_0 - gam x_0,
// x_0 (1 + N gam) = N b_0 - sum_i sum_{j=1..i} b_j, x_i = sum_{k>=i} D_k.
__device__ void cluster_tri_solve_f64(double* v, int lo, int m, int N, double b0, double gam,
                                      double* wsum, double* slot, double* sc) {
  if (lo == 0 && threadIdx.x == 0 && m > 0) v[0] = 0.0;
  __syncthreads();
  double off, tot;
  const double t1 = cta_scan(v, m, false, wsum);
  cluster_prefix(t1, slot, false, &off, &tot);
  double part = 0.0;
  for (int k = threadIdx.x; k < m; k += kSolveThreads) {
    v[k] += off;  // B_i
    part += v[k];
  }
  const double Tl = cta_sum(part, wsum);
  double o2, T;
  cluster_prefix(Tl, slot, false, &o2, &T);
  if (threadIdx.x == 0) {
    const double x0 = (static_cast<double>(N) * b0 - T) / (1.0 + static_cast<double>(N) * gam);
    sc[0] = b0 - gam * x0;
  }
  __syncthreads();
  const double D0 = sc[0];
  for (int k = threadIdx.x; k < m; k += kSolveThreads) v[k] = D0 - v[k];
  __syncthreads();
  const double t3 = cta_scan(v, m, true, wsum);  // suffix sums within the chunk
  double o3, T3;
  cluster_prefix(t3, slot, true, &o3, &T3);  // sums of the chunks after this one
  for (int k = threadIdx.x; k < m; k += kSolveThreads) v[k] += o3;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// k_solve: one cluster of 8 or 16 CTAs solves the new level.
//
// Rank r owns rows [lo, hi).  Four cluster barriers in the common case:
//   A  per-rank totals of the two integer scans -> every rank's offsets
//   B  chunk-edge potentials and fields (neighbour rows of the residual)
//   C  per-rank maxima of |r|, |x|, |b| -> backward error
//   D  keeps every rank's shared memory alive until all remote reads are done
// ---------------------------------------------------------------------------
// Scan segment of the charge grid: s1 = sum of G_i, s2 = sum over the
// segment of the inclusive prefix of G within the segment, len = rows.
// "a then b" is associative: (a1 + b1, a2 + b2 + len_b a1, len_a + len_b).
struct Seg {
  __int128 s2;
  long long s1;
  long long len;
};

// a b as a 128-bit integer from one 64 x 64 -> 128 product (no general
// 128-bit multiplication)
__device__ __forceinline__ __int128 mul_wide(long long a, long long b) {
  const unsigned long long lo = static_cast<unsigned long long>(a) * static_cast<unsigned long long>(b);
  const long long hi = __mul64hi(a, b);
  return static_cast<__int128>((static_cast<unsigned __int128>(static_cast<unsigned long long>(hi)) << 64) | lo);
}

__device__ __forceinline__ Seg seg_then(const Seg& a, const Seg& b) {
  Seg r;
  r.s1 = a.s1 + b.s1;
  r.s2 = a.s2 + b.s2 + mul_wide(b.len, a.s1);
  r.len = a.len + b.len;
  return r;
}

__device__ __forceinline__ Seg shfl_up_seg(const Seg& v, int o) {
  Seg r;
  r.s1 = __shfl_up_sync(0xffffffffu, v.s1, o);
  r.len = __shfl_up_sync(0xffffffffu, v.len, o);
  r.s2 = shfl_up_t(v.s2, o);
  return r;
}

__device__ __forceinline__ Seg shfl_seg(const Seg& v, int src) {
  Seg r;
  r.s1 = __shfl_sync(0xffffffffu, v.s1, src);
  r.len = __shfl_sync(0xffffffffu, v.len, src);
  const unsigned long long lo = static_cast<unsigned long long>(v.s2);
  const unsigned long long hi = static_cast<unsigned long long>(static_cast<unsigned __int128>(v.s2) >> 64);
  const unsigned long long l2 = __shfl_sync(0xffffffffu, lo, src);
  const unsigned long long h2 = __shfl_sync(0xffffffffu, hi, src);
  r.s2 = static_cast<__int128>((static_cast<unsigned __int128>(h2) << 64) | l2);
  return r;
}

// Inclusive warp scan of segments (Kogge-Stone with the "then" operator).
__device__ __forceinline__ Seg warp_scan_seg(Seg v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const Seg y = shfl_up_seg(v, o);
    if (static_cast<int>(lane_id()) >= o) v = seg_then(y, v);
  }
  return v;
}

struct SolveSlotB {
  double first_phi, last_phi, first_E, phi0;
};
struct SolveSlotC {
  unsigned long long rmax, xmax, bmax;  // bit patterns of non-negative doubles
};

// |x| as the bit pattern of a non-negative double: such patterns order like
// the values, so maxima can be taken on the integer pipe (GB300's FP64 pipe
// is narrow).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFULL;
}

// Block maxima of three bit patterns; the result is valid in thread 0.
__device__ void cta_max3(unsigned long long& a, unsigned long long& b, unsigned long long& c,
                         unsigned long long (*red)[32]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
  }
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 0) {
    red[0][w] = a;
    red[1][w] = b;
    red[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kSolveThreads / 32; ++k) {
      a = max(a, red[0][k]);
      b = max(b, red[1][k]);
      c = max(c, red[2][k]);
    }
  }
}

// Circuit charge, surface charge and current of a solved level from the
// circuit scalars of the solve (sc: [2] g, [3] K or Q^n, [6] Q_conv, [7]
// sigma_{n-1}, [8] Q^{n-1}, [9] Q^{n-2}) and the level's phi_0.  strict: a
// circuit whose charge follows Q^n = K - g phi_0^n (series RLC or Tesla).
__device__ __forceinline__ void level_charges(const DevParams* P, const double* sc, bool strict,
                                              double phi0, double* Qn, double* sigma_n, double* I) {
  const double Qconv = sc[6], sigma_prev = sc[7], Q1 = sc[8], Q2 = sc[9];
  if (strict) {
    *Qn = sc[3] - sc[2] * phi0;                             // Eqs. Q4_phi_relation, K_def
    *sigma_n = sigma_prev + (Qconv + *Qn - Q1) * P->inv_A;  // Eq. sigma_update
    *I = (3.0 * *Qn - 4.0 * Q1 + Q2) * P->inv_2dt;
  } else if (P->circuit != CP_CIRCUIT_OPEN) {
    *Qn = sc[3];                                            // weak: the circuit's loop charge
    *sigma_n = sigma_prev + (Qconv + *Qn - Q1) * P->inv_A;  // Eq. top_plate_charge
    *I = (3.0 * *Qn - 4.0 * Q1 + Q2) * P->inv_2dt;
  } else {
    *Qn = Q1;
    *sigma_n = sigma_prev + Qconv * P->inv_A;
    *I = 0.0;
  }
}

// The installed network and the feature window (8 rows of 5 doubles) are
// copied into shared memory while the solve scans (asynchronous copies,
// waited for only when the network runs), so that the predictor reads
// neither from L2 after the solve's last barrier.
__device__ __forceinline__ void prefetch_net(const PredNet* net, PredNet* s_net, const DevState* S,
                                             double* s_feat) {
  const char* src = reinterpret_cast<const char*>(net);
  char* dst = reinterpret_cast<char*>(s_net);
  for (size_t o = 16 * static_cast<size_t>(threadIdx.x); o < kPredNetBytes; o += 16 * kSolveThreads)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst + o))),
                 "l"(src + o)
                 : "memory");
  if (threadIdx.x < kPredWindow * kPredFeat)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(s_feat + threadIdx.x))),
                 "l"(&S->feat[0][0] + threadIdx.x)
                 : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Predictor step on one CTA (all threads), for the paths that keep it in the
// solve: the level's row from the solve's scalars, then the shared predictor
// level (check, ring append, network on the copy in shared memory, s_net).
// (The pointers are passed one by one: a reference to the kernel's parameter
// block would force a copy of it into local memory for the whole solve.)
__device__ __noinline__ void predictor_update(const DevParams* P, DevState* S, const PredNet* s_net,
                                              const double* s_feat, const double* sc, bool strict_rlc,
                                              double phi0) {
  __shared__ PredScratch sp;
  __shared__ PredLevel L;
  const int pos0 = static_cast<int>(sc[37]);
  if (threadIdx.x == 0) {
    double Qn, sigma_n, I;
    level_charges(P, sc, strict_rlc, phi0, &Qn, &sigma_n, &I);
    L.Qconv = sc[6];
    L.phi0 = phi0;
    L.phi0_prev = sc[32];
    L.Qsurf = __dmul_rn(sigma_n, P->area);
    L.Qsurf_prev = __dmul_rn(sc[7], P->area);
    L.Qn = Qn;
    L.Q1 = sc[8];
    L.emitted = sc[33];
    L.ion_eV = sc[34];
    // predictor state loaded with the circuit state at the solve's start
    L.had_pred = (sc[31] != 0.0);
    L.J_pred = sc[30];
    L.err_avg = sc[45];
    L.J_avg = sc[46];
    L.n_eval = static_cast<long long>(sc[47]);
    L.pos = pos0;
    L.n_feat = static_cast<int>(sc[38]);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // this thread's copies of the network
  __syncthreads();
  // the 7 older rows of the window (ring slots pos+1..pos+7, oldest first)
  double v_old = 0.0;
  if (threadIdx.x < kPredIn - kPredFeat)
    v_old = s_feat[((pos0 + 1 + static_cast<int>(threadIdx.x) / kPredFeat) & (kPredWindow - 1)) * kPredFeat +
                   threadIdx.x % kPredFeat];
  pred_level(s_net, P->C, S, &L, v_old, &sp);
}

// The solve of one instance by the CTAs of one cluster (a cluster of one CTA
// in the ensemble launch).
template <typename real>
__device__ __forceinline__ void solve_body(const Bufs& B, int do_push, int mode, double tol) {
  using real2 = typename Pair<real>::type;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = static_cast<int>(cl.block_rank());
  const int nr = static_cast<int>(cl.num_blocks());
  const DevParams* P = B.P;
  DevState* S = B.S;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) Seg wseg[32];
  __shared__ __align__(16) Seg slotA;
  __shared__ __align__(16) Seg s_rank_off;
  __shared__ __align__(16) Seg s_next_off;
  __shared__ __align__(16) __int128 s_U;
  __shared__ double wd[3][32];
  __shared__ unsigned long long wu[3][32];
  __shared__ double s_eta;
  __shared__ SolveSlotB slotB;
  __shared__ SolveSlotC slotC;
  __shared__ double slotd;
  __shared__ double sc[48];
  __shared__ unsigned long long tal[11];  // the push's tallies, read early
  __shared__ int s_stop;
  __shared__ __align__(16) PredNet s_net;  // the network, for the CTA that runs it
  __shared__ __align__(16) double s_feat[kPredWindow * kPredFeat];  // and its feature window

  cudaGridDependencySynchronize();  // the push that deposited G has completed
  if (threadIdx.x == 0) s_stop = (ldcg(&S->status) != 0);
  __syncthreads();
  if (s_stop) return;  // the status cannot change while this kernel runs: all ranks agree

  const int N = P->N;
  const int chunk = (N + nr - 1) / nr;
  const int lo = min(rank * chunk, N);
  const int hi = min(lo + chunk, N);
  const int m = hi - lo;
  long long* Gv = reinterpret_cast<long long*>(smem);  // chunk: G_i of this rank's rows
  double* ph = reinterpret_cast<double*>(smem + align16(8 * chunk));
  double* Ee = ph + chunk;
  double* bb = Ee + chunk;
  double* rr = bb + chunk;

  cudaTriggerProgrammaticLaunchCompletion();
  // the CTA that will run the network fetches it now, behind the scan
  const bool runs_net = (B.net != nullptr && !B.net_in_push && do_push && rank == (nr > 1 ? 1 : 0));
  if (runs_net) prefetch_net(B.net, &s_net, S, s_feat);
  const long long G0 = ldcg(&B.G[0]);
  // G of the next chunk's first row (for the field E_hi of the gather table)
  const long long Gnext = (hi < N) ? ldcg(&B.G[hi]) : 0LL;
  for (int k = threadIdx.x; k < m; k += kSolveThreads) {
    const int i = lo + k;
    const long long g = ldcg(&B.G[i]);
    Gv[k] = (i == 0) ? 0LL : g;  // the prefix S'_i = sum_{j=1..i} G_j leaves G_0 out
    B.Glast[i] = g;
    if (k > 0) B.G[i] = 0;  // a chunk's first row (and G_0) is cleared after barrier A
  }
  const bool last_rows = (hi == N && m > 0);  // this rank owns row N-1 (and node N)
  if (last_rows && threadIdx.x == 0) {
    B.Glast[N] = ldcg(&B.G[N]);
    B.G[N] = 0;
  }
  __syncthreads();
  // circuit row, first part (every rank evaluates the same scalars): the
  // source, the BDF2 history, the circuit solve and the x = 0 row's
  // right-hand side need no scan, so one thread of the last warp does them
  // -- and reads the push's tallies for the commit -- while the CTA scans.
  // Tesla circuit: the last warp forms the new level's loop charges for
  // phi_0 = 0 from the 20 history values (one per lane, warp sums)
  double tq[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (P->circuit == CP_CIRCUIT_TESLA && do_push && threadIdx.x >= kSolveThreads - 32) {
    const int l = static_cast<int>(lane_id());
    const double h = (l < 20) ? ldcg(&S->Qt[l / 5][l % 5]) : 0.0;  // levels n-1..n-4
    const double(*Pm)[20] = (mode == 0) ? P->t_Ps : P->t_Pw;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      double v = (l < 20) ? Pm[i][l] * h : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      tq[i] = v;
    }
  }
  if (threadIdx.x == kSolveThreads - 32) {
    const double qw = P->e * P->weight;
    const long long conv = do_push ? ldcg(&S->conv_count) : 0LL;
    const double Q1 = ldcg(&S->Qh[0]), Q2 = ldcg(&S->Qh[1]);
    const double Q3 = ldcg(&S->Qh[2]);
    // source and BDF2 history of the new level: precomputed by the previous
    // solve except for the first solve of a run
    double Vs, hist;
    if (do_push) {
      Vs = ldcg(&S->nxt_Vs);
      hist = ldcg(&S->nxt_hist);
    } else {
      Vs = B.vs[ldcg(&S->level)];
      const double Q4 = ldcg(&S->Qh[3]);
      hist = P->L4dt2 * (24.0 * Q1 - 22.0 * Q2 + 8.0 * Q3 - Q4) + P->R2dt * (4.0 * Q1 - Q2);
    }
    const double phi0_prev = ldcg(&S->phi0_last);
    // learned weak scheme: the network's prediction of the plasma's change of
    // C phi_0 over this step, used while its tracked error is within bound
    // (the predictor state is loaded in one batch: no chain of dependent loads)
    int pred_ready = 0, feat_pos = 0, n_feat = 0;
    long long n_eval = 0;
    double J_pred = 0.0, err_avg = 0.0, J_avg = 0.0, bound = 0.0;
    double J_fast = 0.0;  // the push formed the usable prediction (FP32 single gap)
    if (B.net != nullptr && B.net_in_push) {
      if (mode == 2) J_fast = ldcg(&S->J_eff);
    } else if (B.net != nullptr) {
      pred_ready = ldcg(&S->pred_ready);
      J_pred = ldcg(&S->J_pred);
      n_eval = ldcg(&S->n_eval);
      err_avg = ldcg(&S->err_avg);
      J_avg = ldcg(&S->J_avg);
      bound = B.net->bound;
      feat_pos = ldcg(&S->feat_pos);
      n_feat = ldcg(&S->n_feat);
    }
    if (!pred_ready) J_pred = 0.0;
    const double J_used =
        (mode == 2 && pred_ready && n_eval >= kPredMinEval && err_avg <= bound * J_avg) ? J_pred : J_fast;
    double g = 0.0, Qpart = Q1, gam = 0.0, inv_den = 1.0;
    if (P->circuit == CP_CIRCUIT_SERIES_RLC) {
      if (mode == 0) {  // strict: Q^n = K - g phi_0^n (Eqs. Q4_phi_relation, K_def)
        g = P->g_strict;
        Qpart = g * (Vs + hist);
        gam = P->gam_strict;
        inv_den = P->inv_den_strict;
      } else {
        // weak (Sec. 2.4.3): the circuit alone, its load capacitor starting
        // from phi_0^{n-1}: a21 Q - hist + phi_0^{n-1} + (Q - Q^{n-1} + J)/C = V_s
        Qpart = (Vs + hist + (Q1 - J_used) * P->inv_C - phi0_prev) * P->g_weak;
      }
    } else if (P->circuit == CP_CIRCUIT_TESLA) {
      // Q1 here is the load capacitor's loop charge Q4^{n-1}
      if (!do_push) {  // level 0: the circuit as it rests before t = 0
        Qpart = Q1;
      } else if (mode == 0) {  // strict: Q4^n = K - [T'^{-1}]_44 phi_0^n
        g = P->t_ws[3];
        Qpart = tq[3];
        gam = P->gam_tesla;
        inv_den = P->inv_den_tesla;
      } else {  // weak: loop 4's capacitor voltage phi_0^{n-1} + (Q4 - Q4^{n-1} + J)/C3
        const double s = (Q1 - J_used) * P->inv_C - phi0_prev;
        Qpart = tq[3] + s * P->t_ww[3];
        sc[36] = s;
      }
      for (int i = 0; i < 5; ++i) sc[40 + i] = tq[i];
    }
    const double Qconv = static_cast<double>(conv) * qw;
    const double sigma_prev = ldcg(&S->sigma);
    // x = 0 row: Eq. Poisson_BC2 (strict) / Eq. Poisson_BC3 (weak), with
    // rho_0 dx^2 / (2 eps0) = alpha G_0 / 2 (G_0 is even: boundary doubling)
    const double b0 = P->dx_eps0 * (sigma_prev + (Qconv + Qpart - Q1) * P->inv_A) +
                      P->alpha * static_cast<double>(G0 / 2);
    sc[0] = b0; sc[1] = gam; sc[2] = g; sc[3] = Qpart; sc[4] = Vs; sc[5] = hist;
    sc[6] = Qconv; sc[7] = sigma_prev; sc[8] = Q1; sc[9] = Q2; sc[10] = Q3;
    sc[12] = static_cast<double>(conv);
    sc[15] = J_used;
    sc[30] = J_pred;
    sc[31] = static_cast<double>(pred_ready);
    sc[32] = phi0_prev;
    sc[35] = inv_den;
    sc[37] = static_cast<double>(feat_pos);  // the predictor's ring slot for this level
    sc[38] = static_cast<double>(n_feat);
    sc[45] = err_avg;  // the predictor's running error averages, updated by its CTA
    sc[46] = J_avg;
    sc[47] = static_cast<double>(n_eval);
    if (do_push) {  // the push's tallies, read before the commit clears them
      sc[33] = static_cast<double>(ldcg(&S->emitted[0]));
      sc[34] = static_cast<double>(ldcg(&S->ion_energy_q)) / 256.0;
      for (int e = 0; e < 2; ++e)
        for (int q = 0; q < kSpecies; ++q) tal[e * kSpecies + q] = ldcg(&S->absorbed[e][q]);
      tal[6] = ldcg(&S->emitted[0]);
      tal[7] = ldcg(&S->emitted[1]);
      tal[8] = ldcg(&S->injected);
      tal[9] = static_cast<unsigned long long>(ldcg(&S->ion_energy_q));
      tal[10] = ldcg(&S->max_cfl_bits);
    } else {
      sc[33] = 0.0;
      sc[34] = 0.0;
      for (int q = 0; q < 11; ++q) tal[q] = 0ULL;
    }
  }
  // this thread's run of rows and its segment totals
  const int per = (m + kSolveThreads - 1) / kSolveThreads;
  const int r0 = min(static_cast<int>(threadIdx.x) * per, m);
  const int r1 = min(r0 + per, m);
  Seg mine;
  mine.s1 = 0;
  mine.s2 = 0;
  mine.len = r1 - r0;
  for (int k = r0; k < r1; ++k) {
    mine.s1 += Gv[k];
    mine.s2 += mine.s1;
  }
  const Seg incl = warp_scan_seg(mine);
  Seg wexcl = shfl_up_seg(incl, 1);  // exclusive within the warp
  if (lane_id() == 0) {
    wexcl.s1 = 0;
    wexcl.s2 = 0;
    wexcl.len = 0;
  }
  const int w = threadIdx.x >> 5;
  if (lane_id() == 31) wseg[w] = incl;
  __syncthreads();
  Seg bexcl;  // everything of this CTA before this warp
  bexcl.s1 = 0;
  bexcl.s2 = 0;
  bexcl.len = 0;
  for (int q = 0; q < w; ++q) bexcl = seg_then(bexcl, wseg[q]);
  // --- barrier A: the CTAs' totals give every rank its offset ----------------
  if (threadIdx.x == 0) {
    Seg tot = bexcl;
    for (int q = w; q < kSolveThreads / 32; ++q) tot = seg_then(tot, wseg[q]);
    slotA = tot;
  }
  cl.sync();
  if (threadIdx.x < 32) {  // lane q reads rank q; a warp scan gives the offsets
    Seg v;
    v.s1 = 0;
    v.s2 = 0;
    v.len = 0;
    if (static_cast<int>(threadIdx.x) < nr) v = *cl.map_shared_rank(&slotA, static_cast<int>(threadIdx.x));
    Seg ci = v;  // inclusive scan over the (at most 8) ranks
#pragma unroll
    for (int o = 1; o < kSolveCtasMax; o <<= 1) {
      const Seg y = shfl_up_seg(ci, o);
      if (static_cast<int>(lane_id()) >= o) ci = seg_then(y, ci);
    }
    Seg ce = shfl_up_seg(ci, 1);
    if (threadIdx.x == 0) {
      ce.s1 = 0;
      ce.s2 = 0;
      ce.len = 0;
    }
    const Seg mine_off = shfl_seg(ce, rank);
    const Seg next_off = shfl_seg(ci, rank);  // everything up to and including this rank
    const Seg all = shfl_seg(ci, nr - 1);
    if (threadIdx.x == 0) {
      s_rank_off = mine_off;
      s_next_off = next_off;
      s_U = all.s2;
      if (m > 0) B.G[lo] = 0;
    }
  }
  __syncthreads();
  const __int128 U = s_U;
  // offset of everything before this thread's run: rank, then warp, then lane
  const Seg off = seg_then(seg_then(s_rank_off, bexcl), wexcl);
  // circuit row, second part: the electrode potential needs the scan total U
  if (threadIdx.x == 0) {
    const double b0 = sc[0], gam = sc[1], inv_den = sc[35];
    const double phi0 = (static_cast<double>(N) * b0 + P->alpha * i128_to_double(U)) * inv_den;
    const double D0 = b0 - gam * phi0;  // D_0 = x_0 - x_1
    sc[11] = D0;
    sc[24] = D0 * P->inv_dx;        // E_0
    sc[25] = P->alpha * P->inv_dx;  // dE_i / dS'_i
  }
  __syncthreads();
  const double b0 = sc[0], gam = sc[1], D0 = sc[11];
  const double alpha = P->alpha, inv_dx = P->inv_dx;
  const double E0 = sc[24], Ea = sc[25];
  // D_i = D_0 + alpha S'_i;  x_i = (N - i) D_0 + alpha (U - P_i);  E_i = D_i / dx
  {
    long long S = off.s1;       // S'_i, running over the run
    __int128 Pex = off.s2;      // P_i = sum_{k<i} S'_k (exclusive)
    for (int k = r0; k < r1; ++k) {
      const int i = lo + k;
      S += Gv[k];
      ph[k] = fma(static_cast<double>(N - i), D0, alpha * i128_to_double(U - Pex));
      Ee[k] = fma(Ea, static_cast<double>(S), E0);
      bb[k] = (i == 0) ? b0 : -alpha * static_cast<double>(Gv[k]);
      Pex += S;
    }
  }
  __syncthreads();

  const bool strict_rlc = (P->circuit == CP_CIRCUIT_SERIES_RLC && mode == 0);
  // the level's charge follows Q^n = K - g phi_0^n (g = 0 at a Tesla level 0)
  const bool strict_c = (P->circuit != CP_CIRCUIT_OPEN) && (mode == 0 || (P->circuit == CP_CIRCUIT_TESLA && !do_push));
  // The neighbouring chunks' edge values follow from the exact prefixes with
  // the same arithmetic their owners use, so no exchange is needed:
  // x_{lo-1} needs P_{lo-1} = P_lo - S'_{lo-1}; x_hi needs P_hi; E_hi needs S'_hi.
  // One thread of four different warps each evaluates one of them.
  double prev_phi, next_phi, nextE, phi0;
  {
    const Seg ro = s_rank_off, no = s_next_off;
    if (threadIdx.x == 0)
      sc[26] = (lo > 0) ? fma(static_cast<double>(N - (lo - 1)), D0,
                              alpha * i128_to_double(U - (ro.s2 - static_cast<__int128>(ro.s1))))
                        : 0.0;
    if (threadIdx.x == 32)
      sc[27] = (hi < N) ? fma(static_cast<double>(N - hi), D0, alpha * i128_to_double(U - no.s2)) : 0.0;
    if (threadIdx.x == 64) sc[28] = (hi < N) ? fma(Ea, static_cast<double>(no.s1 + Gnext), E0) : 0.0;
    if (threadIdx.x == 96) sc[29] = fma(static_cast<double>(N), D0, alpha * i128_to_double(U));  // x_0
    __syncthreads();
    prev_phi = sc[26];
    next_phi = sc[27];
    nextE = sc[28];
    phi0 = sc[29];
  }
  double eta = 0.0;
  double phi0_fin = phi0;  // x_0 after any refinement
  cg::cluster_group::arrival_token done_tok;
  for (int sweep = 0; sweep <= 3; ++sweep) {
    unsigned long long rm = 0ULL, xm = 0ULL, bm = 0ULL;
    for (int k = threadIdx.x; k < m; k += kSolveThreads) {
      const int i = lo + k;
      const double xp = (k + 1 < m) ? ph[k + 1] : next_phi;
      double ri;
      if (i == 0) {
        ri = (1.0 + gam) * ph[k] - xp - bb[k];
      } else {
        const double xq = (k > 0) ? ph[k - 1] : prev_phi;
        ri = (xq - 2.0 * ph[k] + xp) - bb[k];
      }
      rr[k] = ri;
      rm = max(rm, abs_bits(ri));
      xm = max(xm, abs_bits(ph[k]));
    }
    // max |b_i|: on the first pass alpha max |G_i| over rows >= 1 (reduced as
    // an integer) and |b_0|; after a refinement, the bit patterns of |b_i|
    if (sweep == 0) {
      for (int k = threadIdx.x; k < m; k += kSolveThreads)
        if (lo + k > 0) bm = max(bm, static_cast<unsigned long long>(llabs(Gv[k])));
    } else {
      for (int k = threadIdx.x; k < m; k += kSolveThreads) bm = max(bm, abs_bits(bb[k]));
    }
    cta_max3(rm, xm, bm, wu);
    // --- barrier C: backward error over the cluster --------------------------
    if (threadIdx.x == 0) {
      slotC.rmax = rm;
      slotC.xmax = xm;
      slotC.bmax = bm;
    }
    cl.sync();
    if (threadIdx.x < 32) {  // lane q reads rank q
      unsigned long long a = 0, b = 0, c = 0;
      if (static_cast<int>(threadIdx.x) < nr) {
        const SolveSlotC* q = cl.map_shared_rank(&slotC, static_cast<int>(threadIdx.x));
        a = q->rmax;
        b = q->xmax;
        c = q->bmax;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
        c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
      }
      rm = a;
      xm = b;
      bm = c;
    }
    if (threadIdx.x == 0) {
      const double rmd = __longlong_as_double(static_cast<long long>(rm));
      const double xmd = __longlong_as_double(static_cast<long long>(xm));
      const double bmd = (sweep == 0) ? fmax(alpha * static_cast<double>(bm), fabs(b0))
                                      : __longlong_as_double(static_cast<long long>(bm));
      const double nA = fmax(fabs(1.0 + gam) + 1.0, 4.0);
      const double den = nA * xmd + bmd;
      double e = den > 0.0 ? rmd / den : 0.0;
      if (strict_rlc) {  // the circuit row with the potential of row 0
        const double p0 = sweep ? sc[13] : phi0;
        const double Qn = sc[3] - sc[2] * p0;
        const double kvl = P->a21 * Qn - (sc[4] + sc[5]) + p0;
        const double kden = P->a21 * fabs(Qn) + fabs(sc[4] + sc[5]) + fabs(p0);
        if (kden > 0.0) e = fmax(e, fabs(kvl) / kden);
      }
      s_eta = e;
    }
    __syncthreads();
    eta = s_eta;
    if (!(eta > tol) || sweep == 3) {
      done_tok = cl.barrier_arrive();  // this rank's remote reads are done
      break;
    }
    // refinement: solve A delta = r, x -= delta (FP64; rare path)
    const double r0 = (rank == 0) ? rr[0] : 0.0;
    if (rank == 0 && threadIdx.x == 0) sc[14] = r0;
    cl.sync();
    const double r0all = cl.map_shared_rank(&sc[14], 0)[0];
    cluster_tri_solve_f64(rr, lo, m, N, r0all, gam, wd[0], &slotd, sc + 16);
    for (int k = threadIdx.x; k < m; k += kSolveThreads) ph[k] -= rr[k];
    __syncthreads();
    // refined edges: exchange them (rare path)
    if (threadIdx.x == 0 && m > 0) {
      slotB.first_phi = ph[0];
      slotB.last_phi = ph[m - 1];
    }
    cl.sync();
    next_phi = (hi < N) ? cl.map_shared_rank(&slotB, rank + 1)->first_phi : 0.0;
    prev_phi = (lo > 0) ? cl.map_shared_rank(&slotB, rank - 1)->last_phi : 0.0;
    const double phi0_new = cl.map_shared_rank(&slotB, 0)->first_phi;
    for (int k = threadIdx.x; k < m; k += kSolveThreads)
      Ee[k] = (ph[k] - ((k + 1 < m) ? ph[k + 1] : next_phi)) * inv_dx;
    __syncthreads();
    if (threadIdx.x == 0 && m > 0) slotB.first_E = Ee[0];
    cl.sync();
    nextE = (hi < N) ? cl.map_shared_rank(&slotB, rank + 1)->first_E : 0.0;
    sc[13] = phi0_new;
    phi0_fin = phi0_new;
  }

  // outputs; the gather table pairs need the next chunk's first field value
  real2* Epair = reinterpret_cast<real2*>(B.Epair);
  for (int k = threadIdx.x; k < m; k += kSolveThreads) {
    const int i = lo + k;
    B.E64[i] = Ee[k];
    B.phi[i] = ph[k];
    const real e0 = static_cast<real>(Ee[k]);
    const real e1 = (i + 1 < N) ? static_cast<real>((k + 1 < m) ? Ee[k + 1] : nextE) : e0;
    real2 pr;
    pr.x = e0;
    pr.y = e1 - e0;
    Epair[i + 1] = pr;
    if (i == 0) {
      real2 p0;
      p0.x = e0;
      p0.y = real(0);
      Epair[0] = p0;
    }
  }
  if (last_rows && threadIdx.x == 0) B.phi[N] = 0.0;
  // barrier D: no rank leaves (freeing its shared memory) before every
  // rank's remote reads are done
  cl.barrier_wait(std::move(done_tok));
  if (rank == 1) {  // the predictor runs beside rank 0's commit
    if (runs_net) predictor_update(B.P, B.S, &s_net, s_feat, sc, strict_c, phi0_fin);
    return;
  }
  if (rank != 0) return;

  if (threadIdx.x == 0) {
    const int64_t level = S->level + (do_push ? 1 : 0);
    const double dt = P->dt, A = P->area;
    const double phi0 = ph[0];
    const double Qconv = sc[6], Q1 = sc[8], Q2 = sc[9], Q3 = sc[10];
    const long long conv = static_cast<long long>(sc[12]);
    double Qn, sigma_n, I;
    level_charges(P, sc, strict_c, phi0, &Qn, &sigma_n, &I);
    int status = 0;
    if (!isfinite(phi0) || !isfinite(sigma_n) || !isfinite(Qn)) status = CP_ERR_NONFINITE;
    else if (eta > tol) status = CP_ERR_RESIDUAL;

    cp_diag d;
    d.step = level;
    d.t = static_cast<double>(level) * dt;
    d.V_gap = phi0;
    d.I_circ = I;
    d.Q_surf = sigma_n * A;
    d.Q_conv = Qconv;
    d.Q_circ = Qn;
    d.V_source = sc[4];
    d.residual = eta;
    d.ion_energy_eV = static_cast<double>(static_cast<long long>(tal[9])) / 256.0;
    d.max_cfl = static_cast<double>(__uint_as_float(static_cast<unsigned int>(tal[10])));
    d.J_hat = sc[15];
    long long nl[kSpecies];
    for (int s = 0; s < kSpecies; ++s) {
      for (int e = 0; e < 2; ++e) d.absorbed[e][s] = static_cast<int64_t>(tal[e * kSpecies + s]);
      nl[s] = S->n_live[s] - d.absorbed[0][s] - d.absorbed[1][s];
    }
    d.emitted[0] = static_cast<int64_t>(tal[6]);
    d.emitted[1] = static_cast<int64_t>(tal[7]);
    d.injected = static_cast<int64_t>(tal[8]);
    nl[1] += d.injected;
    nl[2] += d.emitted[0] + d.emitted[1];
    for (int s = 0; s < kSpecies; ++s) d.n_live[s] = nl[s];
    d.conv_count = conv;
    S->cur = d;
    if (level < B.hist_rows) B.hist[level] = d;

    // commit the circuit and surface-charge state of the new level
    if (P->circuit == CP_CIRCUIT_TESLA && do_push) {  // the five loop charges
      double Qv[5];
      for (int i = 0; i < 5; ++i)
        Qv[i] = (mode == 0) ? sc[40 + i] - phi0 * P->t_ws[i] : sc[40 + i] + sc[36] * P->t_ww[i];
      for (int k = 3; k > 0; --k)
        for (int i = 0; i < 5; ++i) S->Qt[k][i] = S->Qt[k - 1][i];
      for (int i = 0; i < 5; ++i) S->Qt[0][i] = Qv[i];
      if (!isfinite(Qv[0]) || !isfinite(Qv[1]) || !isfinite(Qv[2]) || !isfinite(Qv[4]))
        status = CP_ERR_NONFINITE;
    }
    S->pv_phi0 = sc[32];  // the predictor's previous level (phi_0, Q_surf)
    S->pv_Qsurf = sc[7] * A;
    S->sigma = sigma_n;
    S->phi0_last = phi0;
    S->Qh[3] = Q3;
    S->Qh[2] = Q2;
    S->Qh[1] = Q1;
    S->Qh[0] = Qn;
    // source and BDF2 history of the next level (off the next solve's critical path)
    S->nxt_Vs = (level + 1 < B.hist_rows + 1) ? B.vs[level + 1] : 0.0;
    S->nxt_hist = P->L4dt2 * (24.0 * Qn - 22.0 * Q1 + 8.0 * Q2 - Q3) + P->R2dt * (4.0 * Qn - Q1);
    S->level = level;
    if (do_push) S->pushed = 1;
    for (int s = 0; s < kSpecies; ++s) {
      S->n_live[s] = nl[s];
      for (int e = 0; e < 2; ++e) S->absorbed[e][s] = 0ULL;
    }
    S->emitted[0] = S->emitted[1] = 0ULL;
    S->injected = 0ULL;
    S->conv_count = 0;
    S->ion_energy_q = 0;
    S->max_cfl_bits = 0u;
    if (status != 0 && S->status == 0) S->status = status;
  }
  // the next push processes the slots in use, rounded up to whole vectors;
  // the padding slots are made dead here
  if (threadIdx.x >= 32 && threadIdx.x < 32 + kSpecies) {
    const int s = threadIdx.x - 32;
    long long na = static_cast<long long>(S->n_alloc[s]);
    if (na > P->cap[s]) na = P->cap[s];
    const long long na4 = (na + 3) & ~3LL;
    real* xs = reinterpret_cast<real*>(S->xi[s]);
    real* us = reinterpret_cast<real*>(S->u[s]);
    for (long long k = na; k < na4; ++k) {
      xs[k] = real(-1);
      us[k] = real(0);
    }
    S->n_alloc[s] = na4;
    S->n_proc[s] = na4;
  }
  if (nr == 1 && runs_net) {  // a one-CTA solve runs the predictor itself
    __syncthreads();
    predictor_update(B.P, B.S, &s_net, s_feat, sc, strict_c, phi0_fin);
  }
}

template <typename real>
__global__ void __launch_bounds__(kSolveThreads, 1) k_solve(Bufs B, int do_push, int mode, double tol) {
  solve_body<real>(B, do_push, mode, tol);
}

// Ensemble: CTA i solves instance i (launched without clusters, so each CTA
// is a cluster of one).
template <typename real>
__global__ void __launch_bounds__(kSolveThreads, 1)
k_solve_ens(const Bufs* __restrict__ Ball, int do_push, int mode, double tol) {
  const Bufs B = Ball[blockIdx.x];
  solve_body<real>(B, do_push, mode, tol);
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
cudaError_t solve_configure(int precision, size_t solve_smem) {
  if (precision == CP_FP32)
    return cudaFuncSetAttribute(k_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(solve_smem));
  return cudaFuncSetAttribute(k_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(solve_smem));
}

size_t solve_smem_bytes(int N, int ctas) {
  const size_t chunk = (N + ctas - 1) / ctas;
  return align16(8 * chunk) + 4 * 8 * chunk;
}

// Largest cluster (16, else 8) the device can run the solve with.
cudaError_t solve_cluster_size(int precision, int N, int* ctas) {
  *ctas = kSolveCtas;
  const void* fn = (precision == CP_FP32) ? reinterpret_cast<const void*>(k_solve<float>)
                                          : reinterpret_cast<const void*>(k_solve<double>);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;
  }
  const size_t smem = solve_smem_bytes(N, kSolveCtasMax);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
      cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kSolveCtasMax, 1, 1);
  cfg.blockDim = dim3(kSolveThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kSolveCtasMax;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) == cudaSuccess && clusters >= 1)
    *ctas = kSolveCtasMax;
  cudaGetLastError();
  return cudaSuccess;
}

cudaError_t solve_ens_configure(int precision, size_t smem) {
  if (precision == CP_FP32)
    return cudaFuncSetAttribute(k_solve_ens<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem));
  return cudaFuncSetAttribute(k_solve_ens<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(smem));
}

cudaError_t solve_ens_launch(int precision, const Bufs* Ball, int n_inst, size_t smem,
                             cudaStream_t st, int do_push, int mode, double tol) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_inst, 1, 1);
  cfg.blockDim = dim3(kSolveThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (precision == CP_FP32) return cudaLaunchKernelEx(&cfg, k_solve_ens<float>, Ball, do_push, mode, tol);
  return cudaLaunchKernelEx(&cfg, k_solve_ens<double>, Ball, do_push, mode, tol);
}

cudaError_t solve_launch(int precision, const Bufs& B, int ctas, size_t smem, cudaStream_t st,
                         int do_push, int mode, double tol) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas, 1, 1);
  cfg.blockDim = dim3(kSolveThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  if (precision == CP_FP32) return cudaLaunchKernelEx(&cfg, k_solve<float>, B, do_push, mode, tol);
  return cudaLaunchKernelEx(&cfg, k_solve<double>, B, do_push, mode, tol);
}

}  // namespace cpk
