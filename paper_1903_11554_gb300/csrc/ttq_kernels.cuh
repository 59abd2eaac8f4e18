// Kernels of one sweep of the dimension-parallel TT cross (Alg. 6 over Alg. 2).
//
// Per sweep, in stream order:
//   k_eval_slabs  evaluate the core entries that are new since the last sweep
//                 (one warp per fiber; node sums V_k on the fly)          [kernel (a)]
//   k_qr          Householder QR of every cross matrix G_k = A(I<=k, I>k),
//                 one CTA per interface                                    [kernel (b)]
//   k_contract    x <- V_1; x <- x G_k^-1; x <- x V_{k+1}: the product of
//                 2d-1 matrices of Sec. 4.1, FP64 or double-double        [kernel (c)]
//   k_samples     Alg. 2, first step: residuals at seeded random positions
//   k_rook_col    Alg. 2, column step: residual on a whole column of the superblock
//   k_rook_row    Alg. 2, row step: residual on a whole row (rook test, Eq. 2)
//   k_update      append the accepted pivots to the nested sets (Alg. 6, end of sweep)
// Every reduction (argmax, sums) runs in a fixed order, so two runs are bitwise equal.
#pragma once
#include "ttq_device.cuh"

namespace ttq {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

// ---------------------------------------------------------------------------
// solves with the QR factors of G_k (one warp; buf/tmp: per-warp shared scratch)

// buf <- G^{-1} buf with factors staged in shared memory: Qs row-major (ld r)
// or, if Qs == nullptr, Q from global; Rs column-major (ld r)
__device__ void warp_col_solve_s(const Dev &D, int k, int r, const double *Qs, const double *Rs,
                                 double *buf, double *tmp) {
  const int lane = lane_id(), ld = D.cap;
  const double *ri = D.rinv[k];
  for (int i = lane; i < r; i += 32) {
    double acc = 0.0;
    if (Qs) for (int b = 0; b < r; ++b) acc = fma(Qs[b * r + i], buf[b], acc);
    else for (int b = 0; b < r; ++b) acc = fma(D.Qr[k][b * ld + i], buf[b], acc);
    tmp[i] = acc;
  }
  __syncwarp();
  for (int j = r - 1; j >= 0; --j) {
    double zj = tmp[j] * ri[j];
    for (int i = lane; i < j; i += 32) tmp[i] = fma(-Rs[i + j * r], zj, tmp[i]);
    if (lane == 0) buf[j] = zj;
    __syncwarp();
  }
}

// core entry Y_k(alpha, i, beta)
__device__ __forceinline__ size_t core_at(const Dev &D, int k, int alpha, int i, int beta) {
  return ((size_t)beta * D.capL[k - 1] + alpha) * D.N[k - 1] + i;
}

// ---------------------------------------------------------------------------
// Argmax of Alg. 2 over the candidates of one interface, spread over the CTAs of
// a kernel.  Every candidate index in [0, count) has its score |E| (-1 if not
// eligible) and E stored in D.cs[k] / D.ce[k].  Pass 1: CTA maxima -> per-interface
// partials -> the last CTA to finish reduces them (deterministic).  Pass 2, in
// that CTA: the first index whose score is within the tie window of the max.
// Returns true in the last CTA (all threads) with the chosen index and E.
__device__ bool cta_pick_last(double myscore, const Dev &D, int k, int count, int *idx_out, double *e_out) {
  __shared__ double sm[TTQ_WARPS];
  __shared__ int si[TTQ_WARPS];
  __shared__ int is_last;
  const int lane = lane_id(), warp = warp_id();
  const int nb = gridDim.x, nw = blockDim.x >> 5;
  __threadfence();                              // publish this thread's candidate writes
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) myscore = fmax(myscore, __shfl_xor_sync(0xffffffffu, myscore, o));
  if (lane == 0) sm[warp] = myscore;
  __syncthreads();
  State *st = D.st;
  if (threadIdx.x == 0) {
    double c = sm[0];
    for (int w = 1; w < nw; ++w) c = fmax(c, sm[w]);
    D.part[(size_t)(k - 1) * nb + blockIdx.x] = c;
    __threadfence();
    unsigned prev = atomicAdd(&st->it[k].counter, 1u);
    is_last = (prev == (unsigned)nb - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double smax = -1.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) smax = fmax(smax, __ldcg(D.part + (size_t)(k - 1) * nb + q));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  if (lane == 0) sm[warp] = smax;
  __syncthreads();
  smax = sm[0];
  for (int w = 1; w < nw; ++w) smax = fmax(smax, sm[w]);
  int first = 0x7fffffff;
  if (smax >= 0.0) {
    const double scale = __longlong_as_double((long long)st->scale_bits);
    const double thr = __dadd_rn(smax, -__dadd_rn(__dmul_rn(TTQ_TIE_REL, smax), __dmul_rn(TTQ_TIE_ABS, scale)));
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
      double v = __ldcg(D.cs[k] + i);
      if (v >= 0.0 && v >= thr) { first = i; break; }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
  __syncthreads();
  if (lane == 0) si[warp] = first;
  __syncthreads();
  first = si[0];
  for (int w = 1; w < nw; ++w) first = min(first, si[w]);
  if (threadIdx.x == 0) st->it[k].counter = 0;
  *idx_out = (first == 0x7fffffff) ? -1 : first;
  *e_out = (first == 0x7fffffff) ? 0.0 : __ldcg(D.ce[k] + first);
  return true;
}

// ---------------------------------------------------------------------------

__global__ void k_setup(Dev *const *Dps) {
  const Dev &D = *Dps[blockIdx.z];
  const int total = D.off[D.d - 1] + D.N[D.d - 1];
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total && D.form == FORM_RN) const_cast<double *>(D.c)[t] = 2.0 * cosh(D.x[t]);
  if (D.uniformT && t < D.N[0]) {
    double th = tanh((D.x[t] - D.x[0]) * 0.5);
    const_cast<double *>(D.T)[t] = th * th;
  }
}

// weighted entries at explicit multi-indices, one warp per point
__global__ void k_eval_points(Dev *const *Dps, const int *idx, long long npts, double *out) {
  const Dev &D = *Dps[blockIdx.z];
  __shared__ int ms[TTQ_WARPS][TTQ_MAXD];
  __shared__ double pl[TTQ_WARPS][TTQ_MAXPAIR];
  const int lane = lane_id(), warp = warp_id();
  long long gw = (long long)blockIdx.x * TTQ_WARPS + warp;
  long long nw = (long long)gridDim.x * TTQ_WARPS;
  for (long long p = gw; p < npts; p += nw) {
    if (lane < D.d) ms[warp][lane] = idx[p * D.d + lane];
    __syncwarp();
    FiberU u = fiber_setup(D, 0, ms[warp], pl[warp]);
    if (lane == 0) out[p] = fiber_value(D, 0, ms[warp], u, pl[warp], ms[warp][0]);
    __syncwarp();
  }
}

// initial index set: the largest |A| among init_samples seeded points
__global__ void k_init(Dev *const *Dps) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  __shared__ int ms[TTQ_WARPS][TTQ_MAXD];
  __shared__ double pl[TTQ_WARPS][TTQ_MAXPAIR];
  __shared__ Best sb[TTQ_WARPS];
  const int lane = lane_id(), warp = warp_id(), d = D.d;
  const unsigned long long sid = stream_id(0, 0, 0);
  Best best = {-1.0, 0x7fffffff, 0.0};
  for (int p = warp; p < D.init_samples; p += TTQ_WARPS) {
    if (lane < d) ms[warp][lane] = draw_index(D.seed, sid, (unsigned long long)p * d + lane, D.N[lane]);
    __syncwarp();
    FiberU u = fiber_setup(D, 0, ms[warp], pl[warp]);
    double v = 0.0;
    if (lane == 0) v = fiber_value(D, 0, ms[warp], u, pl[warp], ms[warp][0]);
    v = __shfl_sync(0xffffffffu, v, 0);
    double s = isfinite(v) ? fabs(v) : -1.0;
    if (better(s, p, best.score, best.idx)) { best.score = s; best.idx = p; best.val = v; }
    __syncwarp();
  }
  best = warp_best(best);
  if (lane == 0) sb[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    Best c = sb[0];
    for (int w = 1; w < TTQ_WARPS; ++w)
      if (better(sb[w].score, sb[w].idx, c.score, c.idx)) c = sb[w];
    sb[0] = c;
    for (int k = 0; k <= d; ++k) { st->r[k] = 1; st->ro[k] = 0; }
    st->sweep = 0; st->status = ST_OK; st->stop = 0; st->nonfinite = 0; st->singular = 0;
    st->nchanges = 0; st->scale_bits = 0ULL; st->value = st->value_lo = st->prev = 0.0;
    st->stop_pending = 0; st->pending_status = 0;
    for (int k = 0; k < TTQ_MAXD; ++k) st->qr_rank[k] = 0;
    st->conv = __longlong_as_double(0x7ff0000000000000LL);
    st->search_evals = 0; st->init_evals = D.init_samples;
    if (!(c.score > 0.0)) { st->status = ST_ERR_NONFINITE; st->stop = 1; }
  }
  __syncthreads();
  // the chosen point: redraw its coordinates
  const int p = sb[0].idx;
  if (threadIdx.x < 32 && lane < d) ms[0][lane] = draw_index(D.seed, sid, (unsigned long long)p * d + lane, D.N[lane]);
  __syncthreads();
  for (int k = 1 + threadIdx.x; k <= d - 1; k += blockDim.x) {
    for (int m = 0; m < d; ++m) {
      D.lidx[k][m] = (m < k) ? ms[0][m] : -1;
      D.ridx[k][m] = (m >= k) ? ms[0][m] : -1;
    }
    D.lpar[k][0] = 0; D.lnode[k][0] = ms[0][k - 1];
    D.rpar[k][0] = 0; D.rnode[k][0] = ms[0][k];
  }
}

// Kernel (a): evaluate every core entry that is new since the previous sweep.
// Fibers (k, alpha, beta) with alpha >= ro[k-1] or beta >= ro[k]; one warp per fiber,
// lanes over the N_k nodes; writes Y_k and the node sums V_k(alpha, beta).
__global__ void __launch_bounds__(TTQ_WARPS * 32) k_eval_slabs(Dev *const *Dps) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  if (st->stop) return;
  __shared__ int ms[TTQ_WARPS][TTQ_MAXD];
  __shared__ double pl[TTQ_WARPS][TTQ_MAXPAIR];
  const int lane = lane_id(), warp = warp_id(), d = D.d;
  // new-fiber counts per mode (lane k-1 <-> mode k), inclusive prefix over modes
  int cnt = 0, rl = 0, rr = 0, ol = 0, orr = 0;
  if (lane < d) {
    rl = st->r[lane]; rr = st->r[lane + 1]; ol = st->ro[lane]; orr = st->ro[lane + 1];
    cnt = rl * rr - ol * orr;
  }
  int pre = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, pre, o);
    if (lane >= o) pre += v;
  }
  const int total = __shfl_sync(0xffffffffu, pre, 31);
  const long long gw = (long long)blockIdx.x * TTQ_WARPS + warp;
  const long long nw = (long long)gridDim.x * TTQ_WARPS;
  double vmax = 0.0;
  int bad = 0;
  unsigned long long fl = 0;
  for (long long g = gw; g < total; g += nw) {
    unsigned ball = __ballot_sync(0xffffffffu, lane < d && pre > g);
    const int km1 = __ffs(ball) - 1;                 // mode k = km1 + 1
    const int k = km1 + 1;
    const int before = __shfl_sync(0xffffffffu, pre - cnt, km1);
    const int Rl = __shfl_sync(0xffffffffu, rl, km1), Rr = __shfl_sync(0xffffffffu, rr, km1);
    const int Ol = __shfl_sync(0xffffffffu, ol, km1), Or = __shfl_sync(0xffffffffu, orr, km1);
    int t = (int)(g - before), alpha, beta;
    const int sizeA = Ol * (Rr - Or);
    if (t < sizeA) { alpha = t / (Rr - Or); beta = Or + t % (Rr - Or); }
    else { t -= sizeA; alpha = Ol + t / Rr; beta = t % Rr; }
    if (lane < d) {
      int v = 0;
      if (lane < k - 1) v = D.lidx[k - 1][alpha * d + lane];
      else if (lane >= k) v = D.ridx[k][beta * d + lane];
      ms[warp][lane] = v;
    }
    __syncwarp();
    FiberU u = fiber_setup(D, km1, ms[warp], pl[warp]);
    const int Nk = D.N[km1];
    fl += (unsigned long long)u.fl_uniform + (unsigned long long)Nk * (u.fl_node + (D.prec ? 20 : 1));
    double *Y = D.Y[k] + core_at(D, k, alpha, 0, beta);
    double s = 0.0;
    dd sd = {0.0, 0.0};
    for (int i = lane; i < Nk; i += 32) {
      double v = fiber_value(D, km1, ms[warp], u, pl[warp], i);
      Y[i] = v;
      if (!isfinite(v)) bad = 1;
      vmax = fmax(vmax, fabs(v));
      if (D.prec) sd = dd_add(sd, {v, 0.0});
      else s += v;
    }
    const size_t vi = (size_t)alpha * D.capL[k] + beta;
    if (D.prec) {
      sd = warp_sum_dd(sd);
      if (lane == 0) { D.V[k][vi] = sd.hi; D.Vlo[k][vi] = sd.lo; }
    } else {
      s = warp_sum(s);
      if (lane == 0) { D.V[k][vi] = s; D.Vlo[k][vi] = 0.0; }
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if (lane == 0 && vmax > 0.0) atomic_max_nonneg(&st->scale_bits, vmax);
  if (__any_sync(0xffffffffu, bad) && lane == 0) st->nonfinite = 1;
  if (lane == 0 && fl) atomicAdd(&st->flops[0], fl);
}

// Kernel (b): QR factors G_k = Q R of every cross matrix G_k = A(I<=k, I>k)
// (r_k x r_k), one CTA per interface.  G_k only grows by bordering: the pivot
// interface k accepted in the previous sweep appends the last row (its new
// element of I<=k) and the last column (its new element of I>k), and nothing
// else changes.  The stored factors are then updated in O(r^2): r - 1 Givens
// rotations fold the new row into R (Q gains a row and a column), and the new
// column of R is Q'^T times the new column of G.  A full Householder QR
// (O(r^3), LAPACK dgeqr2/dorg2r conventions) runs when no factors are stored
// (first sweep, or index sets replaced from outside).
// Stored: Q column-major (Qc) and row-major (Qr), R column- and row-major,
// 1/R_jj; leading dimension cap.

__device__ void qr_store_R(const Dev &D, int k, int r, const double *Rs, int lds, bool rowmajor) {
  const int ld = D.cap;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    int i = e / r, j = e % r;
    double v = (i <= j) ? (rowmajor ? Rs[i * lds + j] : Rs[i + j * lds]) : 0.0;
    D.Rc[k][i + j * ld] = v;
    D.Rr[k][i * ld + j] = v;
  }
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    double rjj = rowmajor ? Rs[j * lds + j] : Rs[j + j * lds];
    if (!(fabs(rjj) > 0.0) || !isfinite(rjj)) D.st->singular = 1;
    D.rinv[k][j] = 1.0 / rjj;
  }
}

__device__ void qr_full(const Dev &D, int k, int r, double *sm) {
  const int ls = r + 1;
  double *G = sm;
  double *tau = sm + (size_t)r * ls;
  const int tid = threadIdx.x, nt = blockDim.x, lane = lane_id(), warp = warp_id();
  for (int e = tid; e < r * r; e += nt) {
    int a = e % r, b = e / r;
    G[a + b * ls] = D.Y[k][core_at(D, k, D.lpar[k][a], D.lnode[k][a], b)];
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (warp == 0) {
      double ss = 0.0;
      for (int i = j + 1 + lane; i < r; i += 32) ss = fma(G[i + j * ls], G[i + j * ls], ss);
      ss = warp_sum(ss);
      double alpha = G[j + j * ls];
      double t = 0.0, beta = alpha, scal = 0.0;
      if (ss > 0.0) {
        double xn = sqrt(ss);
        beta = -copysign(hypot(alpha, xn), alpha);
        t = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      __syncwarp();
      for (int i = j + 1 + lane; i < r; i += 32) G[i + j * ls] *= scal;
      if (lane == 0) { tau[j] = t; G[j + j * ls] = beta; }
    }
    __syncthreads();
    const double tj = tau[j];
    if (tj != 0.0) {
      for (int c = j + 1 + tid; c < r; c += nt) {
        double w = G[j + c * ls];
        for (int i = j + 1; i < r; ++i) w = fma(G[i + j * ls], G[i + c * ls], w);
        w *= tj;
        G[j + c * ls] -= w;
        for (int i = j + 1; i < r; ++i) G[i + c * ls] = fma(-w, G[i + j * ls], G[i + c * ls]);
      }
    }
    __syncthreads();
  }
  qr_store_R(D, k, r, G, ls, false);
  __syncthreads();
  for (int j = r - 1; j >= 0; --j) {
    const double tj = tau[j];
    if (j < r - 1 && tj != 0.0) {
      for (int c = j + 1 + tid; c < r; c += nt) {
        double w = G[j + c * ls];
        for (int i = j + 1; i < r; ++i) w = fma(G[i + j * ls], G[i + c * ls], w);
        w *= tj;
        G[j + c * ls] -= w;
        for (int i = j + 1; i < r; ++i) G[i + c * ls] = fma(-w, G[i + j * ls], G[i + c * ls]);
      }
    }
    __syncthreads();
    for (int i = tid; i < r; i += nt) {
      if (i > j) G[i + j * ls] *= -tj;
      else if (i < j) G[i + j * ls] = 0.0;
    }
    if (tid == 0) G[j + j * ls] = 1.0 - tj;
    __syncthreads();
  }
  const int ld = D.cap;
  for (int e = tid; e < r * r; e += nt) {
    int i = e % r, j = e / r;
    double v = G[i + j * ls];
    D.Qc[k][i + j * ld] = v;
    D.Qr[k][i * ld + j] = v;
  }
}

// factors of the (r-1) x (r-1) leading block are stored; G gained row and column r-1
__device__ void qr_border(const Dev &D, int k, int r, double *sm) {
  const int n = r - 1, ls = r, ld = D.cap;
  double *Rs = sm;                       // r x r row-major
  double *h = Rs + (size_t)r * ls;       // new row of G, reduced by the rotations
  double *cn = h + r;                    // new column of G (length r)
  double *gc = cn + r;                   // rotation cosines
  double *gs = gc + r;                   // rotation sines
  const int tid = threadIdx.x, nt = blockDim.x, lane = lane_id(), warp = warp_id();
  const int anew = D.lpar[k][n], inew = D.lnode[k][n];
  for (int e = tid; e < n * n; e += nt) {
    int i = e / n, j = e % n;
    Rs[i * ls + j] = D.Rr[k][i * ld + j];
  }
  for (int c = tid; c < n; c += nt) h[c] = D.Y[k][core_at(D, k, anew, inew, c)];
  for (int a = tid; a < r; a += nt) cn[a] = D.Y[k][core_at(D, k, D.lpar[k][a], D.lnode[k][a], n)];
  __syncthreads();
  if (warp == 0) {
    for (int j = 0; j < n; ++j) {
      const double x = Rs[j * ls + j], y = h[j];
      double c = 1.0, sn = 0.0, rho = x;
      if (y != 0.0) {
        rho = copysign(hypot(x, y), x);
        const double inv = 1.0 / rho;
        c = x * inv;
        sn = y * inv;
      }
      for (int q = j + 1 + lane; q < n; q += 32) {
        const double t1 = Rs[j * ls + q], t2 = h[q];
        Rs[j * ls + q] = fma(c, t1, sn * t2);
        h[q] = fma(-sn, t1, c * t2);
      }
      if (lane == 0) { Rs[j * ls + j] = rho; h[j] = 0.0; gc[j] = c; gs[j] = sn; }
      __syncwarp();
    }
  }
  __syncthreads();
  // Q' = [[Q, 0], [0, 1]] J_0^T ... J_{n-1}^T, one row per thread
  for (int i = tid; i < r; i += nt) {
    double qlast = (i == n) ? 1.0 : 0.0;
    for (int j = 0; j < n; ++j) {
      const double qa = (i < n) ? D.Qc[k][i + j * ld] : 0.0;
      const double c = gc[j], sn = gs[j];
      D.Qc[k][i + j * ld] = fma(c, qa, sn * qlast);
      qlast = fma(-sn, qa, c * qlast);
    }
    D.Qc[k][i + n * ld] = qlast;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += nt) {
    int i = e / r, j = e % r;
    D.Qr[k][i * ld + j] = D.Qc[k][i + j * ld];
  }
  __syncthreads();
  // new column of R: Q'^T [G(:, n)]
  for (int a = tid; a < r; a += nt) {
    double acc = 0.0;
    for (int i = 0; i < r; ++i) acc = fma(D.Qr[k][i * ld + a], cn[i], acc);
    Rs[a * ls + n] = acc;
  }
  for (int j = tid; j < n; j += nt) Rs[n * ls + j] = 0.0;
  __syncthreads();
  qr_store_R(D, k, r, Rs, ls, true);
}

__global__ void __launch_bounds__(256) k_qr(Dev *const *Dps) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  if (st->stop) return;
  extern __shared__ double sm[];
  const int k = blockIdx.x + 1;
  if (k > D.d - 1) return;                  // instances with fewer interfaces (batches)
  const int r = st->r[k];
  const int have = st->qr_rank[k];
  if (threadIdx.x == 0) {
    IfaceState &I = st->it[k];
    I.active = 0; I.rook_done = 0; I.row = I.col = -1; I.rounds = 0; I.accepted = 0;
    I.err = 0.0; I.evals = 0;
  }
  if (have == r) return;
  if (have >= 1 && have == r - 1) {
    qr_border(D, k, r, sm);
    if (threadIdx.x == 0) atomicAdd(&st->flops[1], (unsigned long long)(12.0 * r * (double)r));
  } else {
    qr_full(D, k, r, sm);
    if (threadIdx.x == 0) atomicAdd(&st->flops[1], (unsigned long long)(8.0 / 3.0 * r * (double)r * r));
  }
  __syncthreads();
  if (threadIdx.x == 0) st->qr_rank[k] = r;
}

// Kernel (c): contraction of the weighted cores with the inverse cross matrices
// (Sec. 4.1): x <- V_1; for k: x <- x G_k^-1 = (Q R^-T x^T)^T; x <- x V_{k+1}.
// One CTA; R_k staged in shared memory for the sequential substitution (one
// warp), the products with Q_k and V_{k+1} spread over all threads.  It only
// feeds the stopping rule, so it runs beside the pivot search; a rule that
// fires is recorded as pending and applied at the end of the sweep.
__global__ void __launch_bounds__(256) k_contract(Dev *const *Dps, int final_dd) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  // per sweep: FP64 contraction for the stopping rule; final_dd: the
  // double-double contraction of the final sets (after the run stopped)
  if (st->stop && !final_dd) return;
  if (final_dd && (!D.prec || st->nonfinite || st->singular)) return;
  const int prec = final_dd;
  extern __shared__ double sm[];
  __shared__ double xh[TTQ_MAXR], xl[TTQ_MAXR], th[TTQ_MAXR], tl[TTQ_MAXR];
  const int tid = threadIdx.x, nt = blockDim.x, lane = lane_id(), warp = warp_id();
  const int d = D.d, ld = D.cap;
  if (st->nonfinite || st->singular) {
    if (tid == 0) {
      st->pending_status = st->nonfinite ? ST_ERR_NONFINITE : ST_ERR_SINGULAR;
      st->stop_pending = 1;
    }
    return;
  }
  double *Rs = sm;                               // r x r row-major
  for (int b = tid; b < st->r[1]; b += nt) { xh[b] = D.V[1][b]; xl[b] = D.Vlo[1][b]; }
  if (tid == 0) {
    unsigned long long fl = 0;
    for (int k = 1; k <= d - 1; ++k) {
      unsigned long long r = st->r[k], rn = st->r[k + 1];
      fl += (3 * r * r + 2 * r * rn) * (prec ? 15 : 1);
    }
    atomicAdd(&st->flops[2], fl);
  }
  for (int k = 1; k <= d - 1; ++k) {
    const int r = st->r[k], rn = st->r[k + 1];
    const double *Qc = D.Qc[k];
    for (int e = tid; e < r * r; e += nt) {
      int i = e / r, j = e % r;
      Rs[i * r + j] = (j >= i) ? D.Rr[k][i * ld + j] : 0.0;
    }
    __syncthreads();
    // forward substitution R^T t = x (one warp, from shared memory)
    if (warp == 0) {
      if (!prec) {
        for (int i = 0; i < r; ++i) {
          double ti = xh[i] * D.rinv[k][i];
          for (int j = i + 1 + lane; j < r; j += 32) xh[j] = fma(-Rs[i * r + j], ti, xh[j]);
          if (lane == 0) th[i] = ti;
          __syncwarp();
        }
      } else {
        for (int i = 0; i < r; ++i) {
          dd ti = dd_div_d({xh[i], xl[i]}, Rs[i * r + i]);
          for (int j = i + 1 + lane; j < r; j += 32) {
            dd v = dd_add({xh[j], xl[j]}, dd_mul_d(ti, -Rs[i * r + j]));
            xh[j] = v.hi; xl[j] = v.lo;
          }
          if (lane == 0) { th[i] = ti.hi; tl[i] = ti.lo; }
          __syncwarp();
        }
      }
    }
    __syncthreads();
    // x <- Q t
    for (int i = tid; i < r; i += nt) {
      if (!prec) {
        double acc = 0.0;
        for (int j = 0; j < r; ++j) acc = fma(Qc[i + j * ld], th[j], acc);
        xh[i] = acc;
      } else {
        dd acc = {0.0, 0.0};
        for (int j = 0; j < r; ++j) acc = dd_add(acc, dd_mul_d({th[j], tl[j]}, Qc[i + j * ld]));
        xh[i] = acc.hi; xl[i] = acc.lo;
      }
    }
    __syncthreads();
    // x <- x V_{k+1}
    for (int b = tid; b < rn; b += nt) {
      if (!prec) {
        double acc = 0.0;
        for (int a = 0; a < r; ++a) acc = fma(xh[a], D.V[k + 1][(size_t)a * D.capL[k + 1] + b], acc);
        th[b] = acc;
      } else {
        dd acc = {0.0, 0.0};
        for (int a = 0; a < r; ++a) {
          size_t vi = (size_t)a * D.capL[k + 1] + b;
          acc = dd_add(acc, dd_mul({xh[a], xl[a]}, {D.V[k + 1][vi], D.Vlo[k + 1][vi]}));
        }
        th[b] = acc.hi; tl[b] = acc.lo;
      }
    }
    __syncthreads();
    for (int b = tid; b < rn; b += nt) { xh[b] = th[b]; xl[b] = tl[b]; }
    __syncthreads();
  }
  if (tid == 0 && final_dd) {
    dd v = dd_mul_d({xh[0], xl[0]}, D.constant);
    st->value = v.hi;
    st->value_lo = v.lo;
    return;
  }
  if (tid == 0) {
    dd v = prec ? dd_mul_d({xh[0], xl[0]}, D.constant) : dd{xh[0] * D.constant, 0.0};
    const double val = v.hi;
    st->value = val;
    st->value_lo = v.lo;
    for (int k = 0; k <= d; ++k) st->ro[k] = st->r[k];
    const int s = st->sweep;
    if (st->rules) {
      if (s > 0) {
        double c = (val != 0.0) ? fabs(val - st->prev) / fabs(val) : fabs(val - st->prev);
        st->conv = c;
        st->changes[st->nchanges & 7] = c;
        st->nchanges++;
      }
      int stop = 0, status = ST_OK;
      if (st->nchanges >= D.conv_window) {
        double mx = 0.0;
        for (int q = 0; q < D.conv_window; ++q) mx = fmax(mx, st->changes[(st->nchanges - 1 - q) & 7]);
        if (mx <= D.tol) { stop = 1; status = ST_OK; }
      }
      if (!stop) {
        int allcap = 1;
        for (int k = 1; k < d; ++k) allcap &= (st->r[k] >= D.cap);
        if (allcap) { stop = 1; status = ST_RANK_CAP; }
      }
      if (!stop && s >= D.max_sweeps - 1) { stop = 1; status = ST_MAX_SWEEPS; }
      if (stop) { st->pending_status = status; st->stop_pending = 1; }
    }
    st->prev = val;
  }
}

// The solve of the next rook step, one CTA per interface with R_k staged in
// shared memory: mode 0 z = G^-1 y for the column step, y = R_{k+1}(:, gamma*);
// mode 1 b = G^-T l for the row step, l = L_k(rho*, :)^T.  Result in zvec[k].
__global__ void __launch_bounds__(256) k_solve(Dev *const *Dps, int mode) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  const int k = blockIdx.x + 1;
  if (k > D.d - 1) return;
  if (st->stop || !st->search) return;
  IfaceState &I = st->it[k];
  if (!I.active || I.rook_done) return;
  extern __shared__ double sm[];
  __shared__ double v[TTQ_MAXR], t[TTQ_MAXR];
  const int tid = threadIdx.x, nt = blockDim.x, lane = lane_id(), warp = warp_id(), ld = D.cap;
  const int r = st->r[k];
  double *Rs = sm;                               // r x r, orientation of the substitution
  double *Qs = D.q_in_smem ? sm + (size_t)r * r : nullptr;   // Q staged too when it fits
  if (mode == 0) {
    const int rn = st->r[k + 1], j = I.col / rn, beta = I.col % rn;
    for (int e = tid; e < r * r; e += nt) {
      int i = e % r, c = e / r;                  // column-major: R[i][c] at Rs[i + c r]
      Rs[i + c * r] = D.Rc[k][i + c * ld];
      if (Qs) Qs[c * r + i] = D.Qr[k][c * ld + i];   // row-major Q[c][i]
    }
    for (int b = tid; b < r; b += nt) v[b] = D.Y[k + 1][core_at(D, k + 1, b, j, beta)];
    __syncthreads();
    for (int i = tid; i < r; i += nt) {          // t = Q^T y
      double acc = 0.0;
      if (Qs) for (int b = 0; b < r; ++b) acc = fma(Qs[b * r + i], v[b], acc);
      else for (int b = 0; b < r; ++b) acc = fma(D.Qr[k][b * ld + i], v[b], acc);
      t[i] = acc;
    }
    __syncthreads();
    if (warp == 0) {                             // back substitution R z = t
      for (int jj = r - 1; jj >= 0; --jj) {
        double zj = t[jj] * D.rinv[k][jj];
        for (int i = lane; i < jj; i += 32) t[i] = fma(-Rs[i + jj * r], zj, t[i]);
        if (lane == 0) v[jj] = zj;
        __syncwarp();
      }
    }
    __syncthreads();
    for (int b = tid; b < r; b += nt) D.zvec[k][b] = v[b];
  } else {
    const int Nk = D.N[k - 1], alpha = I.row / Nk, i0 = I.row % Nk;
    for (int e = tid; e < r * r; e += nt) {
      int i = e / r, c = e % r;                  // row-major: R[i][c] at Rs[i r + c]
      Rs[i * r + c] = D.Rr[k][i * ld + c];
      if (Qs) Qs[i + c * r] = D.Qc[k][i + c * ld];   // column-major Q[i][c]
    }
    for (int b = tid; b < r; b += nt) v[b] = D.Y[k][core_at(D, k, alpha, i0, b)];
    __syncthreads();
    if (warp == 0) {                             // forward substitution R^T t = l
      for (int i = 0; i < r; ++i) {
        double ti = v[i] * D.rinv[k][i];
        for (int jj = i + 1 + lane; jj < r; jj += 32) v[jj] = fma(-Rs[i * r + jj], ti, v[jj]);
        if (lane == 0) t[i] = ti;
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = tid; i < r; i += nt) {          // b = Q t
      double acc = 0.0;
      if (Qs) for (int jj = 0; jj < r; ++jj) acc = fma(Qs[i + jj * r], t[jj], acc);
      else for (int jj = 0; jj < r; ++jj) acc = fma(D.Qc[k][i + jj * ld], t[jj], acc);
      D.zvec[k][i] = acc;
    }
  }
  if (tid == 0) atomicAdd(&st->flops[3], (unsigned long long)(3 * r * r));
}

// shared per-warp scratch of the search kernels
struct SearchSmem {
  int ms[TTQ_WARPS][TTQ_MAXD];
  double pl[TTQ_WARPS][TTQ_MAXPAIR];
  double buf[TTQ_WARPS][TTQ_MAXR];
  double tmp[TTQ_WARPS][TTQ_MAXR];
  int exc[TTQ_WARPS][TTQ_MAXR];
  double z[TTQ_MAXR];
};

// per-warp scratch of the rook kernels (no solve buffers: the solves run in k_solve)
struct RookSmem {
  int ms[TTQ_WARPS][TTQ_MAXD];
  double pl[TTQ_WARPS][TTQ_MAXPAIR];
  int exc[TTQ_WARPS][TTQ_MAXR];
  double z[TTQ_MAXR];
};

__device__ __forceinline__ bool iface_searchable(const Dev &D, const State *st, int k) {
  if (k > D.d - 1) return false;            // instances with fewer interfaces (batches)
  if (st->stop || !st->search) return false;
  const int rk = st->r[k];
  if (rk >= D.cap) return false;
  if (st->r[k - 1] * D.N[k - 1] <= rk) return false;
  if (D.N[k] * st->r[k + 1] <= rk) return false;
  return true;
}

// Alg. 2, first step: residuals E = A - B_k R_{k+1} at seeded random positions.
__global__ void __launch_bounds__(TTQ_WARPS * 32) k_samples(Dev *const *Dps) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  const int k = blockIdx.y + 1;
  if (!iface_searchable(D, st, k)) return;
  __shared__ SearchSmem sh;
  extern __shared__ double fac[];
  const int lane = lane_id(), warp = warp_id(), d = D.d;
  const int rk = st->r[k], rl = st->r[k - 1], rn = st->r[k + 1];
  const int Nk = D.N[k - 1], Nk1 = D.N[k];
  const int M = rl * Nk, Ncol = Nk1 * rn, S = D.S[k];
  double *Rs = fac;                                  // R column-major, ld rk
  double *Qs = D.q_in_smem ? fac + (size_t)rk * rk : nullptr;   // Q row-major, ld rk
  for (int e = threadIdx.x; e < rk * rk; e += blockDim.x) {
    int i = e % rk, c = e / rk;
    Rs[i + c * rk] = D.Rc[k][i + c * D.cap];
    if (Qs) Qs[c * rk + i] = D.Qr[k][c * D.cap + i];
  }
  __syncthreads();
  const unsigned long long sid = stream_id(st->sweep, k, 1);
  double best = -1.0;
  long long evals = 0;
  unsigned long long fl = 0;
  for (int t = blockIdx.x * TTQ_WARPS + warp; t < S; t += gridDim.x * TTQ_WARPS) {
    const int rho = draw_index(D.seed, sid, 2ULL * t, (unsigned long long)M);
    const int gam = draw_index(D.seed, sid, 2ULL * t + 1, (unsigned long long)Ncol);
    bool ex = false;
    for (int a = lane; a < rk; a += 32) {
      if (D.lpar[k][a] * Nk + D.lnode[k][a] == rho) ex = true;
      if (D.rnode[k][a] * rn + D.rpar[k][a] == gam) ex = true;
    }
    if (__any_sync(0xffffffffu, ex)) {
      if (lane == 0) { D.cs[k][t] = -1.0; D.ce[k][t] = 0.0; }
      continue;
    }
    const int alpha = rho / Nk, i = rho % Nk, j = gam / rn, beta = gam % rn;
    if (lane < d) {
      int v;
      if (lane < k - 1) v = D.lidx[k - 1][alpha * d + lane];
      else if (lane == k - 1) v = i;
      else if (lane == k) v = j;
      else v = D.ridx[k + 1][beta * d + lane];
      sh.ms[warp][lane] = v;
    }
    // y = R_{k+1}(:, gamma) = Y_{k+1}(:, j, beta)
    for (int b = lane; b < rk; b += 32) sh.buf[warp][b] = D.Y[k + 1][core_at(D, k + 1, b, j, beta)];
    __syncwarp();
    FiberU u = fiber_setup(D, k - 1, sh.ms[warp], sh.pl[warp]);
    double A = 0.0;
    if (lane == 0) A = fiber_value(D, k - 1, sh.ms[warp], u, sh.pl[warp], i);
    A = __shfl_sync(0xffffffffu, A, 0);
    warp_col_solve_s(D, k, rk, Qs, Rs, sh.buf[warp], sh.tmp[warp]);
    double acc = 0.0;
    for (int b = lane; b < rk; b += 32) acc = fma(D.Y[k][core_at(D, k, alpha, i, b)], sh.buf[warp][b], acc);
    acc = warp_sum(acc);
    const double E = A - acc;
    const double sc = isfinite(E) ? fabs(E) : -1.0;
    if (lane == 0) { D.cs[k][t] = sc; D.ce[k][t] = E; }
    best = fmax(best, sc);
    ++evals;
    fl += (unsigned long long)(u.fl_uniform + u.fl_node) + 3ULL * rk * rk + 2ULL * rk + 1;
    __syncwarp();
  }
  if (lane == 0 && evals) atomicAdd(&st->it[k].evals, (unsigned long long)evals);
  if (lane == 0 && fl) atomicAdd(&st->flops[3], fl);
  int pick;
  double epick;
  if (!cta_pick_last(best, D, k, S, &pick, &epick)) return;
  if (pick < 0) return;                        // nothing to search from
  if (threadIdx.x == 0) {
    const int t = pick;
    IfaceState &I = st->it[k];
    I.row = draw_index(D.seed, sid, 2ULL * t, (unsigned long long)M);
    I.col = draw_index(D.seed, sid, 2ULL * t + 1, (unsigned long long)Ncol);
    I.err = epick;
    I.active = 1;
  }
}

// Alg. 2, column step: E(:, gamma*) over all rows rho = (alpha, i); argmax -> rho*.
__global__ void __launch_bounds__(TTQ_WARPS * 32, 3) k_rook_col(Dev *const *Dps) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  const int k = blockIdx.y + 1;
  if (k > D.d - 1) return;
  if (st->stop || !st->search) return;
  IfaceState &I = st->it[k];
  if (!I.active || I.rook_done) return;
  __shared__ RookSmem sh;
  const int lane = lane_id(), warp = warp_id(), d = D.d;
  const int rk = st->r[k], rl = st->r[k - 1], rn = st->r[k + 1];
  const int Nk = D.N[k - 1];
  const int gam = I.col, j = gam / rn, beta = gam % rn;
  for (int b = threadIdx.x; b < rk; b += blockDim.x) sh.z[b] = D.zvec[k][b];
  __syncthreads();
  const int nch = (Nk + TTQ_CHUNK - 1) / TTQ_CHUNK;
  const int items = rl * nch;
  double best = -1.0;
  long long evals = 0;
  unsigned long long fl = 0;
  for (int w = blockIdx.x * TTQ_WARPS + warp; w < items; w += gridDim.x * TTQ_WARPS) {
    const int alpha = w / nch, ch = w % nch;
    if (lane < d) {
      int v = 0;
      if (lane < k - 1) v = D.lidx[k - 1][alpha * d + lane];
      else if (lane == k) v = j;
      else if (lane > k) v = D.ridx[k + 1][beta * d + lane];
      sh.ms[warp][lane] = v;
    }
    // rows of the cross with this parent alpha: excluded nodes i
    int nex = 0;
    for (int a0 = 0; a0 < rk; a0 += 32) {
      int a = a0 + lane;
      bool hit = a < rk && D.lpar[k][a] == alpha;
      unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (hit) sh.exc[warp][nex + __popc(bal & ((1u << lane) - 1))] = D.lnode[k][a];
      nex += __popc(bal);
    }
    __syncwarp();
    FiberU u = fiber_setup(D, k - 1, sh.ms[warp], sh.pl[warp]);
    const int i0 = ch * TTQ_CHUNK, i1 = min(Nk, i0 + TTQ_CHUNK);
    fl += (unsigned long long)u.fl_uniform + (unsigned long long)(i1 - i0) * (u.fl_node + 2 * rk + 1);
    // each lane takes 4 nodes of the chunk at once: 4 independent loads per step
    // of the product L_k(rho, :) z over the core
    int iq[4];
    bool ok[4];
    double A[4], acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      iq[q] = i0 + lane + 32 * q;
      bool ex = false;
      for (int e = 0; e < nex; ++e) ex |= (sh.exc[warp][e] == iq[q]);
      ok[q] = iq[q] < i1 && !ex;
      A[q] = ok[q] ? fiber_value(D, k - 1, sh.ms[warp], u, sh.pl[warp], iq[q]) : 0.0;
      acc[q] = 0.0;
    }
    {
      const double *Yc = D.Y[k] + core_at(D, k, alpha, 0, 0);
      const size_t cst = (size_t)D.capL[k - 1] * Nk;
      const int c0 = min(iq[0], Nk - 1), c1 = min(iq[1], Nk - 1), c2 = min(iq[2], Nk - 1), c3 = min(iq[3], Nk - 1);
#pragma unroll 4
      for (int b = 0; b < rk; ++b) {
        const double zb = sh.z[b];
        const double *row = Yc + b * cst;
        acc[0] = fma(row[c0], zb, acc[0]);
        acc[1] = fma(row[c1], zb, acc[1]);
        acc[2] = fma(row[c2], zb, acc[2]);
        acc[3] = fma(row[c3], zb, acc[3]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (iq[q] >= i1) continue;
      const int rho = alpha * Nk + iq[q];
      if (!ok[q]) { D.cs[k][rho] = -1.0; D.ce[k][rho] = 0.0; continue; }
      const double E = A[q] - acc[q];
      const double sc = isfinite(E) ? fabs(E) : -1.0;
      D.cs[k][rho] = sc;
      D.ce[k][rho] = E;
      best = fmax(best, sc);
      ++evals;
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
  if (lane == 0 && evals) atomicAdd(&I.evals, (unsigned long long)evals);
  if (lane == 0 && fl) atomicAdd(&st->flops[4], fl);
  int pick;
  double epick;
  if (!cta_pick_last(best, D, k, rl * Nk, &pick, &epick)) return;
  if (threadIdx.x == 0) {
    if (pick < 0) I.active = 0;
    else I.row = pick;
  }
}

// Alg. 2, row step: E(rho*, :) over all columns gamma = (j, beta); argmax -> gamma_new,
// then the rook test (Eq. 2): gamma_new == gamma* ends the search.
__global__ void __launch_bounds__(TTQ_WARPS * 32, 3) k_rook_row(Dev *const *Dps) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  const int k = blockIdx.y + 1;
  if (k > D.d - 1) return;
  if (st->stop || !st->search) return;
  IfaceState &I = st->it[k];
  if (!I.active || I.rook_done) return;
  __shared__ RookSmem sh;
  const int lane = lane_id(), warp = warp_id(), d = D.d;
  const int rk = st->r[k], rn = st->r[k + 1];
  const int Nk = D.N[k - 1], Nk1 = D.N[k];
  const int rho = I.row, alpha = rho / Nk, i = rho % Nk;
  for (int b = threadIdx.x; b < rk; b += blockDim.x) sh.z[b] = D.zvec[k][b];
  __syncthreads();
  const int nch = (Nk1 + TTQ_CHUNK - 1) / TTQ_CHUNK;
  const int items = rn * nch;
  double best = -1.0;
  unsigned long long fl = 0;
  long long evals = 0;
  for (int w = blockIdx.x * TTQ_WARPS + warp; w < items; w += gridDim.x * TTQ_WARPS) {
    const int beta = w / nch, ch = w % nch;
    if (lane < d) {
      int v = 0;
      if (lane < k - 1) v = D.lidx[k - 1][alpha * d + lane];
      else if (lane == k - 1) v = i;
      else if (lane > k) v = D.ridx[k + 1][beta * d + lane];
      sh.ms[warp][lane] = v;
    }
    int nex = 0;
    for (int b0 = 0; b0 < rk; b0 += 32) {
      int b = b0 + lane;
      bool hit = b < rk && D.rpar[k][b] == beta;
      unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (hit) sh.exc[warp][nex + __popc(bal & ((1u << lane) - 1))] = D.rnode[k][b];
      nex += __popc(bal);
    }
    __syncwarp();
    FiberU u = fiber_setup(D, k, sh.ms[warp], sh.pl[warp]);
    const int j0 = ch * TTQ_CHUNK, j1 = min(Nk1, j0 + TTQ_CHUNK);
    fl += (unsigned long long)u.fl_uniform + (unsigned long long)(j1 - j0) * (u.fl_node + 2 * rk + 1);
    int jq[4];
    bool ok[4];
    double A[4], acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      jq[q] = j0 + lane + 32 * q;
      bool ex = false;
      for (int e = 0; e < nex; ++e) ex |= (sh.exc[warp][e] == jq[q]);
      ok[q] = jq[q] < j1 && !ex;
      A[q] = ok[q] ? fiber_value(D, k, sh.ms[warp], u, sh.pl[warp], jq[q]) : 0.0;
      acc[q] = 0.0;
    }
    {
      const double *Yr = D.Y[k + 1] + core_at(D, k + 1, 0, 0, beta);
      const int c0 = min(jq[0], Nk1 - 1), c1 = min(jq[1], Nk1 - 1), c2 = min(jq[2], Nk1 - 1), c3 = min(jq[3], Nk1 - 1);
#pragma unroll 4
      for (int a = 0; a < rk; ++a) {
        const double za = sh.z[a];
        const double *row = Yr + (size_t)a * Nk1;
        acc[0] = fma(row[c0], za, acc[0]);
        acc[1] = fma(row[c1], za, acc[1]);
        acc[2] = fma(row[c2], za, acc[2]);
        acc[3] = fma(row[c3], za, acc[3]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (jq[q] >= j1) continue;
      const int g = jq[q] * rn + beta;
      if (!ok[q]) { D.cs[k][g] = -1.0; D.ce[k][g] = 0.0; continue; }
      const double E = A[q] - acc[q];
      const double sc = isfinite(E) ? fabs(E) : -1.0;
      D.cs[k][g] = sc;
      D.ce[k][g] = E;
      best = fmax(best, sc);
      ++evals;
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
  if (lane == 0 && evals) atomicAdd(&I.evals, (unsigned long long)evals);
  if (lane == 0 && fl) atomicAdd(&st->flops[5], fl);
  int pick;
  double epick;
  if (!cta_pick_last(best, D, k, Nk1 * rn, &pick, &epick)) return;
  if (threadIdx.x == 0) {
    if (pick < 0) {
      I.active = 0;
    } else {
      const int rounds = I.rounds + 1;
      const bool done = (pick == I.col) || rounds >= D.rook_max;
      I.rounds = rounds;
      I.col = pick;
      I.err = epick;
      I.rook_done = done ? 1 : 0;
    }
  }
}

// End of sweep (Alg. 6): append every accepted pivot, nested by construction.
// Inside the whole-run graph it also sets the WHILE condition: continue while
// the run is not over, never past max_sweeps (every path reaches the end).
__global__ void k_update(Dev *const *Dps, cudaGraphConditionalHandle h, int use_cond) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  const int d = D.d;
  const int k = threadIdx.x + 1;            // one thread per interface (d - 1 <= 31)
  __shared__ int rold[TTQ_MAXD + 1];
  __shared__ int nacc;
  __shared__ long long ev;
  __shared__ int mode;                      // 0: nothing to do, 1: apply pending stop, 2: no search, 3: append
  if (threadIdx.x == 0) {
    nacc = 0; ev = 0;
    if (st->stop) mode = 0;
    else if (st->stop_pending) mode = 1;
    else if (!st->search) mode = 2;
    else mode = 3;
  }
  __syncthreads();
  if (mode == 1 && threadIdx.x == 0) { st->stop = 1; st->status = st->pending_status; }
  if (mode == 2 && threadIdx.x == 0) st->sweep++;
  if (mode == 3) {
    for (int q = threadIdx.x; q <= d; q += blockDim.x) rold[q] = st->r[q];
    __syncthreads();
    const double scale = __longlong_as_double((long long)st->scale_bits);
    if (k <= d - 1) {
      IfaceState &I = st->it[k];
      atomicAdd((unsigned long long *)&ev, (unsigned long long)I.evals);
      if (I.active) {
        const bool acc = fabs(I.err) > D.pivot_tol * scale && rold[k] < D.cap;
        I.accepted = acc ? 1 : 0;
        if (acc) {
          atomicAdd(&nacc, 1);
          const int Nk = D.N[k - 1], rn = rold[k + 1];
          const int alpha = I.row / Nk, i = I.row % Nk, j = I.col / rn, beta = I.col % rn;
          const int a = rold[k];
          int *L = D.lidx[k] + (size_t)a * d, *R = D.ridx[k] + (size_t)a * d;
          for (int m = 0; m < d; ++m) {
            L[m] = (m < k - 1) ? D.lidx[k - 1][alpha * d + m] : (m == k - 1 ? i : -1);
            R[m] = (m == k) ? j : (m > k ? D.ridx[k + 1][beta * d + m] : -1);
          }
          D.lpar[k][a] = alpha; D.lnode[k][a] = i;
          D.rpar[k][a] = beta; D.rnode[k][a] = j;
        }
      }
    }
    __syncthreads();
    if (k <= d - 1 && st->it[k].accepted) st->r[k] = rold[k] + 1;
    if (threadIdx.x == 0) {
      st->search_evals += ev;
      if (st->rules && nacc == 0) { st->stop = 1; st->status = ST_NO_PIVOT; }
      st->sweep++;
    }
  }
  if (use_cond && threadIdx.x == 0) {
    const int guard = ++st->loop_guard;
    const int cont = !st->stop && st->sweep < D.max_sweeps && guard < D.max_sweeps + 2;
    cudaGraphSetConditional(h, cont ? 1u : 0u);
  }
}

__global__ void k_begin(Dev *const *Dps, int sweep, int rules, int search) {
  State *st = Dps[blockIdx.z]->st;
  st->sweep = sweep;
  st->rules = rules;
  st->search = search;
  st->stop_pending = 0;
  st->loop_guard = 0;
  if (!rules) st->stop = 0;
}

// End of a batched sweep inside the whole-run graph: continue while any
// instance of the batch is still running (bounded by the largest max_sweeps).
__global__ void k_batch_cond(Dev *const *Dps, int count, int max_sweeps, unsigned *guard,
                             cudaGraphConditionalHandle h) {
  int running = 0;
  for (int q = threadIdx.x; q < count; q += blockDim.x) running |= !Dps[q]->st->stop;
  running = __syncthreads_or(running);
  if (threadIdx.x == 0) {
    const unsigned g = ++(*guard);
    cudaGraphSetConditional(h, (running && g < (unsigned)max_sweeps + 2) ? 1u : 0u);
  }
}

}  // namespace ttq
