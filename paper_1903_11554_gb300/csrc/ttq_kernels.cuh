// Kernels of one sweep of the dimension-parallel TT cross (Alg. 6 over Alg. 2).
//
// Per sweep, in stream order:
//   k_eval_slabs  evaluate the core entries that are new since the last sweep
//                 (fibers split into rows of 32 nodes; node sums V_k)     [kernel (a)]
//   k_qr_row,     QR factors of every cross matrix G_k = A(I<=k, I>k), one CTA
//   k_qr          per interface: bordering by the new row (beside kernel (a))
//                 and the new column, full Householder when none stored [kernel (b)]
//   k_contract    x <- V_1; x <- x G_k^-1; x <- x V_{k+1}: the product of
//                 2d-1 matrices of Sec. 4.1, FP64 or double-double        [kernel (c)]
//   k_samples     Alg. 2, first step: residuals at seeded random positions
//   k_rook_col    Alg. 2, column step: residual on a whole column of the superblock
//   k_solve       argmax pass 2, search state, the next step's solve
//   k_rook_row    Alg. 2, row step: residual on a whole row (rook test, Eq. 2)
//   k_solve       ... and, the last one, the end of the sweep: the accepted
//                 pivots appended to the nested sets (Alg. 6), ranks, stopping rules
// Every reduction (argmax, sums) runs in a fixed order, so two runs are bitwise equal.
#pragma once
#include "ttq_device.cuh"

namespace ttq {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

// ---------------------------------------------------------------------------
// Stage r x r blocks of the QR factors in shared memory: for e = (row, col) in
// [0, r)^2, a_dst[row * ldd + col] = a_src[row * ld + col], the same for b if
// b_dst; whole CTA, with eight independent loads in flight per thread (the
// copies are latency bound).
__device__ __forceinline__ void stage_block(double *a_dst, const double *a_src, double *b_dst,
                                            const double *b_src, int r, int ld, int ldd) {
  const int n = r * r, nt = blockDim.x;
  for (int e0 = threadIdx.x; e0 < n; e0 += 4 * nt) {
    double va[4], vb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * nt;
      if (e < n) {
        const int o = (e / r) * ld + e % r;
        va[u] = a_src[o];
        if (b_dst) vb[u] = b_src[o];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * nt;
      if (e < n) {
        const int o = (e / r) * ldd + e % r;
        a_dst[o] = va[u];
        if (b_dst) b_dst[o] = vb[u];
      }
    }
  }
}
__device__ __forceinline__ void stage_compact(double *a_dst, const double *a_src, double *b_dst,
                                              const double *b_src, int r, int ld) {
  stage_block(a_dst, a_src, b_dst, b_src, r, ld, r);
}

// asynchronous global -> shared copies (cp.async, 8 bytes each)
__device__ __forceinline__ void cp_async8(double *smem, const double *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// the same r x r copies as stage_compact, issued asynchronously: a warp per
// row, lanes over its columns (no index division on the issuing path)
__device__ __forceinline__ void stage_compact_async(double *a_dst, const double *a_src, double *b_dst,
                                                    const double *b_src, int r, int ld) {
  const int lane = lane_id(), nw = blockDim.x >> 5;
  for (int row = warp_id(); row < r; row += nw) {
    const size_t so = (size_t)row * ld;
    const int dof = row * r;
    for (int c = lane; c < r; c += 32) {
      cp_async8(a_dst + dof + c, a_src + so + c);
      if (b_dst) cp_async8(b_dst + dof + c, b_src + so + c);
    }
  }
}

// out[i] = sum_b M(i, b) x[b], i < r, with M(i, b) at Mp[i * si + b * sb]; the
// sum over b split into parts over all threads, partial sums combined in order
__device__ __forceinline__ void cta_gemv(const double *Mp, int si, int sb, const double *x, int r, double *part,
                                        double *out) {
  const int nt = blockDim.x, P = r <= 64 ? 4 : 2, rows = nt / P;
  const int i = threadIdx.x % rows, pp = threadIdx.x / rows;
  if (i < r && pp < P) {
    const int b0 = pp * r / P, b1 = (pp + 1) * r / P;
    double acc = 0.0;
    for (int b = b0; b < b1; ++b) acc = fma(Mp[(size_t)i * si + (size_t)b * sb], x[b], acc);
    part[pp * TTQ_MAXR + i] = acc;
  }
  __syncthreads();
  if (threadIdx.x < r) {
    double acc = part[threadIdx.x];
    for (int q = 1; q < P; ++q) acc += part[q * TTQ_MAXR + threadIdx.x];
    out[threadIdx.x] = acc;
  }
  __syncthreads();
}

// Substitutions with the scaled triangles, one warp, lane l holding entries
// l + 32 q in registers.  Back: v <- t, then for j = r-1 .. 0: v_i -= C_ij v_j
// (i < j), C = R D^-1 column-major; the result z = D^-1 v.  Forward: u <- l,
// then for i = 0 .. r-1: u_m -= S_im u_i (m > i), S = D^-1 R row-major; the
// result t = D^-1 u.  The steps are split into segments of 32 so that the
// number of register blocks a step touches is a compile-time constant (an FP64
// warp instruction costs its full time whether or not its lanes are active).
template <int NQ>
__device__ __forceinline__ void back_step(int j, const double (&c)[NQ], double *tq, double *vout) {
  const int lane = lane_id();
  const double vj = __shfl_sync(0xffffffffu, tq[NQ - 1], j & 31);
  if (lane == (j & 31)) vout[j] = vj;
#pragma unroll
  for (int q = NQ - 1; q >= 0; --q)               // the block the next step reads first
    if (q < NQ - 1 || lane + 32 * q < j) tq[q] = fma(-c[q], vj, tq[q]);
}
// the entries of column j the step uses (the others are never read)
template <int NQ>
__device__ __forceinline__ void back_load(const double *C, int ld, int j, double (&c)[NQ]) {
  const int lane = lane_id();
#pragma unroll
  for (int q = 0; q < NQ; ++q) c[q] = (q < NQ - 1 || lane + 32 * q < j) ? C[lane + 32 * q + (size_t)j * ld] : 0.0;
}
// four steps at a time with their triangle entries loaded first, so that no
// load sits on the chain of multiply-adds and shuffles
template <int NQ>
__device__ __forceinline__ void back_seg(const double *C, int ld, int jhi, int jlo, double *tq, double *vout) {
  int jj = jhi;
  for (; jj - 3 >= jlo; jj -= 4) {
    double c0[NQ], c1[NQ], c2[NQ], c3[NQ];
    back_load<NQ>(C, ld, jj, c0);
    back_load<NQ>(C, ld, jj - 1, c1);
    back_load<NQ>(C, ld, jj - 2, c2);
    back_load<NQ>(C, ld, jj - 3, c3);
    back_step<NQ>(jj, c0, tq, vout);
    back_step<NQ>(jj - 1, c1, tq, vout);
    back_step<NQ>(jj - 2, c2, tq, vout);
    back_step<NQ>(jj - 3, c3, tq, vout);
  }
  for (; jj >= jlo; --jj) {
    double c0[NQ];
    back_load<NQ>(C, ld, jj, c0);
    back_step<NQ>(jj, c0, tq, vout);
  }
}
// vout[j] = v_j after the back substitution (z = D^-1 vout); C column-major, leading dimension ld
__device__ __forceinline__ void warp_back_subst(const double *C, const double *t, double *vout, int r, int ld) {
  const int lane = lane_id(), nq = (r + 31) >> 5;
  double tq[TTQ_MAXR / 32];
#pragma unroll
  for (int q = 0; q < TTQ_MAXR / 32; ++q) tq[q] = (lane + 32 * q < r) ? t[lane + 32 * q] : 0.0;
  for (int sg = nq; sg >= 1; --sg) {
    const int jhi = min(r, 32 * sg) - 1, jlo = 32 * (sg - 1);
    switch (sg) {
      case 4: back_seg<4>(C, ld, jhi, jlo, tq, vout); break;
      case 3: back_seg<3>(C, ld, jhi, jlo, tq, vout); break;
      case 2: back_seg<2>(C, ld, jhi, jlo, tq, vout); break;
      default: back_seg<1>(C, ld, jhi, jlo, tq, vout); break;
    }
  }
}
// Forward substitution in reversed row order: lane l, block q holds row
// m = r - 1 - (l + 32 q), so the rows a step still updates (m > i) fill the
// low blocks and a step touches ceil((r - 1 - i) / 32) register blocks, as in
// the back substitution, instead of every block from i's on.
template <int NQ>
__device__ __forceinline__ void fwd_load(const double *S, int r, int ld, int jj, double (&c)[NQ]) {
  const int lane = lane_id();
  const double *Si = S + (size_t)(r - 1 - jj) * ld + (r - 1);
#pragma unroll
  for (int q = 0; q < NQ; ++q) c[q] = (q < NQ - 1 || lane + 32 * q < jj) ? Si[-(lane + 32 * q)] : 0.0;
}
template <int NQ>
__device__ __forceinline__ void fwd_step(int r, int jj, const double (&c)[NQ], double *vq, double *uout) {
  const int lane = lane_id();
  const double ui = __shfl_sync(0xffffffffu, vq[NQ - 1], jj & 31);
  if (lane == (jj & 31)) uout[r - 1 - jj] = ui;
#pragma unroll
  for (int q = NQ - 1; q >= 0; --q)
    if (q < NQ - 1 || lane + 32 * q < jj) vq[q] = fma(-c[q], ui, vq[q]);
}
template <int NQ>
__device__ __forceinline__ void fwd_seg(const double *S, int r, int ld, int jhi, int jlo, double *vq, double *uout) {
  int jj = jhi;                                  // jj = r - 1 - i, i ascending
  for (; jj - 3 >= jlo; jj -= 4) {
    double c0[NQ], c1[NQ], c2[NQ], c3[NQ];
    fwd_load<NQ>(S, r, ld, jj, c0);
    fwd_load<NQ>(S, r, ld, jj - 1, c1);
    fwd_load<NQ>(S, r, ld, jj - 2, c2);
    fwd_load<NQ>(S, r, ld, jj - 3, c3);
    fwd_step<NQ>(r, jj, c0, vq, uout);
    fwd_step<NQ>(r, jj - 1, c1, vq, uout);
    fwd_step<NQ>(r, jj - 2, c2, vq, uout);
    fwd_step<NQ>(r, jj - 3, c3, vq, uout);
  }
  for (; jj >= jlo; --jj) {
    double c0[NQ];
    fwd_load<NQ>(S, r, ld, jj, c0);
    fwd_step<NQ>(r, jj, c0, vq, uout);
  }
}
// uout[i] = u_i after the forward substitution (t = D^-1 uout); S row-major, leading dimension ld
__device__ __forceinline__ void warp_fwd_subst(const double *S, const double *l, double *uout, int r, int ld) {
  const int lane = lane_id(), nq = (r + 31) >> 5;
  double vq[TTQ_MAXR / 32];
#pragma unroll
  for (int q = 0; q < TTQ_MAXR / 32; ++q) vq[q] = (lane + 32 * q < r) ? l[r - 1 - (lane + 32 * q)] : 0.0;
  for (int sg = nq; sg >= 1; --sg) {
    const int jhi = min(r, 32 * sg) - 1, jlo = 32 * (sg - 1);
    switch (sg) {
      case 4: fwd_seg<4>(S, r, ld, jhi, jlo, vq, uout); break;
      case 3: fwd_seg<3>(S, r, ld, jhi, jlo, vq, uout); break;
      case 2: fwd_seg<2>(S, r, ld, jhi, jlo, vq, uout); break;
      default: fwd_seg<1>(S, r, ld, jhi, jlo, vq, uout); break;
    }
  }
}

// Node chunks of a mode for the rook steps: the ceil(N/32) rows of 32 nodes split
// as evenly as possible into nch = ceil(rows / R) chunks of at most R rows (R in
// 1, 2, 4), so no chunk is a nearly empty one that still costs full warp
// instructions.
struct NodeChunks {
  int nch, base, extra;
};
__device__ __forceinline__ NodeChunks node_chunks(int N, int R) {
  const int rows = (N + 31) >> 5, nch = (rows + R - 1) / R;
  return {nch, rows / nch, rows % nch};
}
// nodes [i0, i1) of chunk ch, in nq rows of 32
__device__ __forceinline__ void chunk_span(const NodeChunks &c, int ch, int N, int &i0, int &i1, int &nq) {
  const int q0 = ch * c.base + min(ch, c.extra);
  nq = c.base + (ch < c.extra ? 1 : 0);
  i0 = 32 * q0;
  i1 = min(N, 32 * (q0 + nq));
}

// Rows per work item of a step (the same in every CTA): the smallest power of two
// up to Rmax whose items all fit in one wave of the grid's warps.  An item's latency is
// its FP64 instruction count (each takes its scheduler's FP64 unit for a fixed
// time), so small items finish a low-rank step early, while full-rank steps use
// 4-row items to spread the fibers' shared setup.  outer: lane k-1 holds
// interface k's outer rank (0 when the interface does not search), Nl its nodes.
__device__ __forceinline__ int rows_per_item(int outer, int Nl, int Rmax = 4) {
  const long long warps = (long long)gridDim.x * TTQ_WARPS;
  int R = 1;
  for (; R < Rmax; R *= 2) {
    long long items = outer ? (long long)outer * node_chunks(Nl, R).nch : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) items += __shfl_xor_sync(0xffffffffu, items, o);
    if (items <= warps) break;
  }
  return R;
}

// core entry Y_k(alpha, i, beta)
__device__ __forceinline__ size_t core_at(const Dev &D, int k, int alpha, int i, int beta) {
  return ((size_t)beta * D.capL[k - 1] + alpha) * D.N[k - 1] + i;
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

// Initial nested sets: r0 multi-indices taken from init_samples seeded random
// points in decreasing |A| (ties by draw order), a point kept when its first
// and last node indices differ from those of the points already kept (so all
// its prefixes and suffixes are new and every interface gets rank r0); a point
// whose value is not finite and nonzero ends the scan.  I<=k = the kept
// points' prefixes of length k and I>k = their suffixes from mode k+1, in the
// order kept: nested by construction (Eq. 4).  Fewer than r0 usable points:
// status NONFINITE.
__global__ void k_init(Dev *const *Dps) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  __shared__ int ms[TTQ_WARPS][TTQ_MAXD];
  __shared__ double pl[TTQ_WARPS][TTQ_MAXPAIR];
  __shared__ double score[TTQ_MAX_INIT];          // |A| of each point (-1: not finite), -2 once consumed
  __shared__ int first[TTQ_MAX_INIT], lastc[TTQ_MAX_INIT];   // its first and last node index
  __shared__ int chosen[TTQ_MAXR];
  __shared__ int nchosen, pick;
  __shared__ double rs[TTQ_WARPS];
  __shared__ int ri[TTQ_WARPS];
  const int lane = lane_id(), warp = warp_id(), d = D.d, ns = D.init_samples;
  const unsigned long long sid = stream_id(0, 0, 0);
  for (int p = warp; p < ns; p += TTQ_WARPS) {
    if (lane < d) ms[warp][lane] = draw_index(D.seed, sid, (unsigned long long)p * d + lane, D.N[lane]);
    __syncwarp();
    FiberU u = fiber_setup(D, 0, ms[warp], pl[warp]);
    double v = 0.0;
    if (lane == 0) v = fiber_value(D, 0, ms[warp], u, pl[warp], ms[warp][0]);
    v = __shfl_sync(0xffffffffu, v, 0);
    if (lane == 0) {
      score[p] = isfinite(v) ? fabs(v) : -1.0;
      first[p] = ms[warp][0];
      lastc[p] = ms[warp][d - 1];
    }
    __syncwarp();
  }
  if (threadIdx.x == 0) nchosen = 0;
  __syncthreads();
  // greedy scan in decreasing |A|: one block-wide argmax (ties to the lowest
  // draw) per point consumed
  for (int it = 0; it < ns; ++it) {
    double bv = -3.0;
    int bi = 0x7fffffff;
    for (int p = threadIdx.x; p < ns; p += blockDim.x)
      if (score[p] > bv || (score[p] == bv && p < bi)) { bv = score[p]; bi = p; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { rs[warp] = bv; ri[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = rs[0];
      int q = ri[0];
      for (int w = 1; w < TTQ_WARPS; ++w)
        if (rs[w] > v || (rs[w] == v && ri[w] < q)) { v = rs[w]; q = ri[w]; }
      pick = (v > 0.0) ? q : -1;                    // no finite nonzero point left: stop
      if (pick >= 0) {
        bool fresh = true;
        for (int c = 0; c < nchosen; ++c)
          fresh &= first[chosen[c]] != first[pick] && lastc[chosen[c]] != lastc[pick];
        if (fresh) chosen[nchosen++] = pick;
        score[pick] = -2.0;
      }
    }
    __syncthreads();
    if (pick < 0 || nchosen >= D.r0) break;
  }
  const int r0 = nchosen;
  if (threadIdx.x == 0) {
    const int rr = r0 >= 1 ? r0 : 1;
    for (int k = 0; k <= d; ++k) { st->r[k] = (k == 0 || k == d) ? 1 : rr; st->ro[k] = 0; }
    st->sweep = 0; st->status = ST_OK; st->stop = 0; st->nonfinite = 0; st->singular = 0;
    st->nchanges = 0; st->scale_bits = 0ULL; st->value = st->value_lo = st->prev = 0.0;
    st->stop_pending = 0; st->pending_status = 0; st->search_abort = 0; st->seq_k = 0; st->seq_nacc = 0;
    for (int k = 0; k < TTQ_MAXD; ++k) { st->qr_rank[k] = 0; st->qr_row[k] = 0; }
    st->conv = __longlong_as_double(0x7ff0000000000000LL);
    st->search_evals = 0; st->init_evals = D.init_samples;
    if (r0 < D.r0) { st->status = ST_ERR_NONFINITE; st->stop = 1; }
  }
  if (r0 < 1) return;
  // the kept points' node indices, redrawn: ms-like rows per point in chosen order
  for (int e = threadIdx.x; e < r0 * d; e += blockDim.x) {
    const int j = e / d, m = e % d;
    const int x = draw_index(D.seed, sid, (unsigned long long)chosen[j] * d + m, D.N[m]);
    for (int k = 1; k <= d - 1; ++k) {
      D.lidx[k][j * d + m] = (m < k) ? x : -1;
      D.ridx[k][j * d + m] = (m >= k) ? x : -1;
    }
    // I<=k[j] = (I<=k-1[j], x_j[k-1]) and I>k[j] = (x_j[k], I>k+1[j]); the empty
    // sets I<=0 and I>d have the single row 0
    if (m <= d - 2) { D.lnode[m + 1][j] = x; D.lpar[m + 1][j] = m == 0 ? 0 : j; }
    if (m >= 1) { D.rnode[m][j] = x; D.rpar[m][j] = m == d - 1 ? 0 : j; }
  }
}

// Kernel (a): evaluate every core entry that is new since the previous sweep.
// Fibers (k, alpha, beta) with alpha >= ro[k-1] or beta >= ro[k]; a work item is a
// chunk of 1, 2, 4 .. rows of 32 nodes of a fiber, up to the whole fiber (one warp,
// lanes over the nodes; the smallest rows per item whose items fit one wave of
// the grid), so a low-rank sweep's few fibers still spread over many warps.
// Writes Y_k; the warp that completes a fiber (an atomic count of its rows) forms
// the node sum V_k(alpha, beta) from the written entries, lane l adding nodes
// l, l + 32, .. and the lanes combined by the fixed butterfly -- the same order
// whatever the chunking.
__global__ void __launch_bounds__(TTQ_WARPS * 32) k_eval_slabs(Dev *const *Dps) {
  __shared__ Dev sD;
  extern __shared__ double dyn_t[];
  const Dev &D = stage_dev(Dps, sD);
  const double *Ts = stage_pair_table(D, dyn_t);
  __syncthreads();
  pdl_wait();
  // the successor (kernel b) is released at the end, not here: launched early
  // its CTAs would take the resident slots left free for the QR row kernel
  State *st = D.st;
  if (st->stop) return;
  __shared__ int ms[TTQ_WARPS][TTQ_MAXD];
  __shared__ double pl[TTQ_WARPS][TTQ_MAXPAIR];
  const int lane = lane_id(), warp = warp_id(), d = D.d;
  // new-fiber counts per mode (lane k-1 <-> mode k)
  int cnt = 0, rl = 0, rr = 0, ol = 0, orr = 0, Nl = 1;
  if (lane < d) {
    rl = st->r[lane]; rr = st->r[lane + 1]; ol = st->ro[lane]; orr = st->ro[lane + 1];
    cnt = rl * rr - ol * orr;
    Nl = D.N[lane];
  }
  const int R = rows_per_item(cnt, Nl, 32);
  const int nchl = node_chunks(Nl, R).nch;
  const int icnt = cnt * nchl;                   // items of mode lane+1
  int pre = icnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, pre, o);
    if (lane >= o) pre += v;
  }
  const int total = __shfl_sync(0xffffffffu, pre, 31);
  const long long nw = (long long)gridDim.x * TTQ_WARPS;
  double vmax = 0.0;
  int bad = 0;
  unsigned long long fl = 0;
  for (long long g = (long long)deal_slot(warp, D.sms, total) * gridDim.x + blockIdx.x; g < total; g += nw) {
    unsigned ball = __ballot_sync(0xffffffffu, lane < d && pre > g);
    const int km1 = __ffs(ball) - 1;                 // mode k = km1 + 1
    const int k = km1 + 1;
    const int before = __shfl_sync(0xffffffffu, pre - icnt, km1);
    const int Cn = __shfl_sync(0xffffffffu, cnt, km1);
    const int Rr = __shfl_sync(0xffffffffu, rr, km1);
    const int Ol = __shfl_sync(0xffffffffu, ol, km1), Or = __shfl_sync(0xffffffffu, orr, km1);
    const int local = (int)(g - before);
    const int ch = local / Cn;                       // chunk-major walk
    int t = local % Cn, alpha, beta;
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
    FiberU u = fiber_setup(D, km1, ms[warp], pl[warp], Ts);
    const int Nk = D.N[km1], nrows = (Nk + 31) >> 5;
    const NodeChunks nc = node_chunks(Nk, R);
    int i0, i1, nq;
    chunk_span(nc, ch, Nk, i0, i1, nq);
    fl += (unsigned long long)u.fl_uniform + (unsigned long long)(i1 - i0) * (u.fl_node + (D.prec ? 5 : 1));
    double *Y = D.Y[k] + core_at(D, k, alpha, 0, beta);
    const size_t fib = (size_t)alpha * D.capL[k] + beta;
    for (int q = 0; q < nq; ++q) {
      const int i = i0 + 32 * q + lane;
      if (i < i1) {
        const double v = fiber_value(D, km1, ms[warp], u, pl[warp], i);
        Y[i] = v;
        if (!isfinite(v)) bad = 1;
        vmax = fmax(vmax, fabs(v));
      }
    }
    // the warp that completes the fiber forms its node sum
    int last = 0;
    if (nq == nrows) {
      last = 1;                                      // whole fiber in this item
    } else {
      __threadfence();
      __syncwarp();
      if (lane == 0) {
        const unsigned old = atomicAdd(D.vcnt[k] + fib, (unsigned)nq);
        last = (old + nq == (unsigned)nrows) ? 1 : 0;
        if (last) D.vcnt[k][fib] = 0;
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last) __threadfence();
    }
    if (last) {
      __syncwarp();
      if (D.prec) {
        // Neumaier-compensated sum of the lane's nodes (running sum s, and c the
        // sum of its exact rounding errors), then the lanes' pairs added in
        // the butterfly with each addition's exact error carried along: V +
        // Vlo is the node sum to ~N u^2 relative
        double sn = 0.0, cn = 0.0;
        for (int i = lane; i < Nk; i += 32) {
          const double x = __ldcg(Y + i), t = sn + x;
          cn += (fabs(sn) >= fabs(x)) ? ((sn - t) + x) : ((x - t) + sn);
          sn = t;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double so = __shfl_xor_sync(0xffffffffu, sn, o), co = __shfl_xor_sync(0xffffffffu, cn, o);
          // lower lane's value first, so every lane forms the same pair
          const dd e = ((lane & o) == 0) ? two_sum(sn, so) : two_sum(so, sn);
          sn = e.hi;
          cn = ((lane & o) == 0) ? (cn + co) + e.lo : (co + cn) + e.lo;
        }
        const dd sd = fast_two_sum(sn, cn);
        if (lane == 0) { D.V[k][fib] = sd.hi; D.Vlo[k][fib] = sd.lo; }
      } else {
        double sr = 0.0;
        for (int i = lane; i < Nk; i += 32) sr += __ldcg(Y + i);
        sr = warp_sum(sr);
        if (lane == 0) { D.V[k][fib] = sr; D.Vlo[k][fib] = 0.0; }
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if (lane == 0 && vmax > 0.0) atomic_max_nonneg(&st->scale_bits, vmax);
  if (__any_sync(0xffffffffu, bad) && lane == 0) st->nonfinite = 1;
  if (lane == 0 && fl) atomicAdd(&st->flops[0], fl);
  pdl_release();
}

// Kernel (b), second half: QR factors G_k = Q R of every cross matrix
// G_k = A(I<=k, I>k) (r_k x r_k), one CTA per interface.  G_k only grows by bordering: the pivot
// interface k accepted in the previous sweep appends the last row (its new
// element of I<=k) and the last column (its new element of I>k), and nothing
// else changes.  The stored factors are then updated in O(r^2): r - 1 plane
// rotations fold the new row into R (Q gains a row and a column), and the new
// column of R is Q'^T times the new column of G.  A full Householder QR
// (O(r^3), LAPACK dgeqr2/dorg2r conventions) runs when no factors are stored
// (first sweep, or index sets replaced from outside).  With several pivots per
// sweep (MULTI) an interface may append m > 1 rows and columns: one bordering
// update (row, then column) per appended pair, in append order.
// Stored: Q column-major (Qc) and row-major (Qr), R column- and row-major,
// 1/R_jj, and R with its diagonal divided out for the FP64 substitutions:
// Cc = R D^-1 column-major (entries R_ij / R_jj, back substitution) and
// Sr = D^-1 R row-major (entries R_ij / R_ii, forward substitution), D = diag R,
// so each step of a substitution is one multiply-add on its dependency chain;
// leading dimension cap.

__device__ void qr_store_R(const Dev &D, int k, int r, const double *Rs, int lds, bool rowmajor) {
  __shared__ double rinv_s[TTQ_MAXR];
  const int ld = D.cap;
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    double rjj = rowmajor ? Rs[j * lds + j] : Rs[j + j * lds];
    if (!(fabs(rjj) > 0.0) || !isfinite(rjj)) D.st->singular = 1;
    rinv_s[j] = 1.0 / rjj;
    D.rinv[k][j] = rinv_s[j];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    int i = e / r, j = e % r;
    double v = (i <= j) ? (rowmajor ? Rs[i * lds + j] : Rs[i + j * lds]) : 0.0;
    D.Rc[k][i + j * ld] = v;
    D.Rr[k][i * ld + j] = v;
    if (i < j) {
      D.Cc[k][i + j * ld] = v * rinv_s[j];
      D.Sr[k][i * ld + j] = rinv_s[i] * v;
    }
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

// Factors of the (r-1) x (r-1) leading block are stored; G gained row and
// column n = r-1.  Appending the row h (the new row over the old columns) to R
// takes the rotations J_j (rows j and n) that zero h_0 .. h_{n-1} in turn.
// Their parameters follow from p = R^-T h without the sequential chain of the
// rotations themselves: with t_j^2 = 1 + sum_{i<=j} p_i^2 (t_{-1} = 1),
// c_j = t_{j-1} / t_j and s_j = p_j / t_j, since the entry J_j zeroes is
// R_jj p_j / t_{j-1} (Gill, Golub, Murray & Saunders 1974, method C1, for the
// update R^T R + h h^T).  p comes from the row solve of the search that found
// the pivot when it is still at hand, else from a forward substitution.  The
// rotations then run down every column of R and every row of Q independently.
// The row append needs only entries evaluated in earlier sweeps (the new row's
// parent alpha* belongs to the old left set), so it runs beside kernel (a) on
// the second stream: qr_border_row leaves the rotated n x n block of R in Rr and
// Q' = [[Q, 0], [0, 1]] J_0^T .. J_{n-1}^T in Qc / Qr.  qr_border_col then
// adds the new column of R, Q'^T G(:, n), from the new slab of the core.
__device__ void qr_border_row(const Dev &D, int k, int r, double *sm) {
  IfaceState &I = D.st->it[k];
  const int n = r - 1, ls = r, ld = D.cap;
  double *Rs = sm;                       // r x r row-major (ld ls)
  double *h = Rs + (size_t)r * ls;       // new row of G over the old columns
  double *gc = h + r;                    // rotation cosines
  double *gs = gc + r;                   // rotation sines
  double *p = gs + r;                    // R^-T h
  double *ri = p + r;                    // 1 / R_jj of the old factor
  const int tid = threadIdx.x, nt = blockDim.x, lane = lane_id(), warp = warp_id();
  const int anew = D.lpar[k][n], inew = D.lnode[k][n];
  const bool cached = I.prank == n && I.prow == anew * D.N[k - 1] + inew;
  stage_block(Rs, D.Rr[k], nullptr, nullptr, n, ld, ls);
  for (int c = tid; c < n; c += nt) {
    h[c] = D.Y[k][core_at(D, k, anew, inew, c)];
    ri[c] = D.rinv[k][c];
    if (cached) p[c] = D.pvec[k][c];
  }
  __syncthreads();
  if (warp == 0) {
    if (!cached) {                         // R^T p = h, the same scaled substitution as the row solve
      warp_fwd_subst(D.Sr[k], h, p, n, ld);
      __syncwarp();
      for (int c = lane; c < n; c += 32) p[c] *= ri[c];
      __syncwarp();
    }
    // t_j by an inclusive scan of p_j^2 over chunks of 32, then c_j and s_j
    double carry = 1.0;
    for (int base = 0; base < n; base += 32) {
      const int j = base + lane;
      const double pj = (j < n) ? p[j] : 0.0;
      double sc = pj * pj;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, sc, o);
        if (lane >= o) sc += y;
      }
      const double tj = sqrt(carry + sc);
      double tp = __shfl_up_sync(0xffffffffu, tj, 1);
      if (lane == 0) tp = sqrt(carry);
      if (j < n) {
        const double inv = 1.0 / tj;
        gc[j] = tp * inv;
        gs[j] = pj * inv;
      }
      carry += __shfl_sync(0xffffffffu, sc, 31);
    }
  }
  __syncthreads();
  if (tid < 128) {
    // column q of R: rotations 0 .. q (the last one makes the diagonal entry)
    for (int q = tid; q < n; q += 128) {
      double hq = h[q];
      for (int j = 0; j <= q; ++j) {
        const double c = gc[j], sn = gs[j], rjq = Rs[j * ls + q];
        Rs[j * ls + q] = fma(c, rjq, sn * hq);
        hq = fma(-sn, rjq, c * hq);
      }
    }
  } else {
    // Q' one row per thread, old Q read sixteen columns at a time
    for (int i = tid - 128; i < r; i += nt - 128) {
      double qlast = (i == n) ? 1.0 : 0.0;
      for (int j0 = 0; j0 < n; j0 += 16) {
        double qa[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) qa[u] = (i < n && j0 + u < n) ? D.Qc[k][i + (j0 + u) * ld] : 0.0;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int j = j0 + u;
          if (j < n) {
            const double c = gc[j], sn = gs[j];
            const double q = fma(c, qa[u], sn * qlast);
            qlast = fma(-sn, qa[u], c * qlast);
            D.Qc[k][i + j * ld] = q;
            D.Qr[k][i * ld + j] = q;
          }
        }
      }
      D.Qc[k][i + n * ld] = qlast;
      D.Qr[k][i * ld + n] = qlast;
    }
  }
  __syncthreads();
  // the rotated n x n block of R in every stored layout (the column append
  // leaves it as it is and only adds the last column): 1/R_jj first
  for (int j = tid; j < n; j += nt) {
    const double rjj = Rs[j * ls + j];
    if (!(fabs(rjj) > 0.0) || !isfinite(rjj)) D.st->singular = 1;
    ri[j] = 1.0 / rjj;
    D.rinv[k][j] = ri[j];
  }
  __syncthreads();
  // row-major layouts a warp per row, column-major ones a warp per column, so
  // every store of a warp is contiguous
  const int nw = nt >> 5;
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j < n; j += 32) {
      const double v = (i <= j) ? Rs[i * ls + j] : 0.0;
      D.Rr[k][i * ld + j] = v;
      if (i < j) D.Sr[k][i * ld + j] = ri[i] * v;
    }
  for (int j = warp; j < n; j += nw)
    for (int i = lane; i < n; i += 32) {
      const double v = (i <= j) ? Rs[i * ls + j] : 0.0;
      D.Rc[k][i + j * ld] = v;
      if (i < j) D.Cc[k][i + j * ld] = v * ri[j];
    }
}

// second half of the bordering update: new column of R = Q'^T G(:, n), written
// into every stored layout beside the block the row append stored
__device__ void qr_border_col(const Dev &D, int k, int r, double *sm, double *part) {
  const int n = r - 1, ld = D.cap, tid = threadIdx.x, nt = blockDim.x;
  double *cn = sm;                       // new column of G (length r)
  double *v = cn + r;                    // Q'^T cn
  for (int a = tid; a < r; a += nt) cn[a] = D.Y[k][core_at(D, k, D.lpar[k][a], D.lnode[k][a], n)];
  __syncthreads();
  cta_gemv(D.Qr[k], 1, ld, cn, r, part, v);   // v[a] = sum_i Q'[i][a] cn[i]
  const double rnn = v[n];
  if (tid == 0 && (!(fabs(rnn) > 0.0) || !isfinite(rnn))) D.st->singular = 1;
  const double rinn = 1.0 / rnn;
  if (tid == 0) D.rinv[k][n] = rinn;
  for (int a = tid; a <= n; a += nt) {
    const double va = v[a];
    D.Rc[k][a + n * ld] = va;
    D.Rr[k][a * ld + n] = va;
    if (a < n) {
      D.Cc[k][a + n * ld] = va * rinn;
      D.Sr[k][a * ld + n] = D.rinv[k][a] * va;
      D.Rc[k][n + a * ld] = 0.0;             // below the diagonal
      D.Rr[k][n * ld + a] = 0.0;
    }
  }
}

// Kernel (b), first half: the row append of every interface whose G_k grew by
// one (second stream, beside kernel (a)).
__global__ void __launch_bounds__(256) k_qr_row(Dev *const *Dps) {
  __shared__ Dev sD;
  const Dev &D = stage_dev(Dps, sD);
  State *st = D.st;
  if (st->stop) return;
  extern __shared__ double sm[];
  const int k = blockIdx.x + 1;
  if (k > D.d - 1) return;
  const int r = st->r[k], have = st->qr_rank[k];
  if (!(have >= 1 && have == r - 1)) return;
  qr_border_row(D, k, r, sm);
  if (threadIdx.x == 0) st->qr_row[k] = r;
}

template <bool MULTI>
__global__ void __launch_bounds__(256) k_qr(Dev *const *Dps) {
  __shared__ Dev sD;
  const Dev &D = stage_dev(Dps, sD);
  // the run flag, the rank and the factors' rank were written in earlier
  // sweeps, the row append's mark by k_qr_row (a full dependency of this
  // launch): read before the wait for kernel (a)
  State *st = D.st;
  const int k = blockIdx.x + 1;
  const bool mine = k <= D.d - 1;           // instances with fewer interfaces (batches)
  const int stop = st->stop;
  const int r = mine ? st->r[k] : 0;
  const int have = mine ? st->qr_rank[k] : 0;
  const int rowdone = mine ? st->qr_row[k] : 0;
  pdl_wait();
  pdl_release();
  if (stop || !mine) return;
  extern __shared__ double sm[];
  if (threadIdx.x < (MULTI ? D.npiv : 1)) {
    IfaceState &I = search_state(D, st, k, threadIdx.x);
    I.active = 0; I.rook_done = 0; I.row = I.col = -1; I.rounds = 0; I.accepted = 0;
    I.err = 0.0; I.evals = 0; I.smax_bits = 0ULL; I.stage_count = 0; I.items_done = 0; I.epoch = 0;
    I.acc_arrive = 0; I.merged = 0;
  }
  if (have == r) {
    if (threadIdx.x == 0) st->it[k].prank = -1;
    return;
  }
  __shared__ double part[4 * TTQ_MAXR];
  if (have >= 1 && have == r - 1 && rowdone == r) {
    qr_border_col(D, k, r, sm, part);
    if (threadIdx.x == 0) atomicAdd(&st->flops[1], (unsigned long long)(12.0 * r * (double)r));
  } else if (MULTI && have >= 1) {
    // several pivots appended in the last sweep: one bordering update per new
    // row and column, in append order (the rows' entries over the new columns
    // come from this sweep's kernel (a), which precedes this kernel)
    for (int t = have + 1; t <= r; ++t) {
      qr_border_row(D, k, t, sm);
      __syncthreads();
      qr_border_col(D, k, t, sm, part);
      __syncthreads();
      if (threadIdx.x == 0) atomicAdd(&st->flops[1], (unsigned long long)(12.0 * t * (double)t));
    }
  } else {
    qr_full(D, k, r, sm);
    if (threadIdx.x == 0) atomicAdd(&st->flops[1], (unsigned long long)(8.0 / 3.0 * r * (double)r * r));
  }
  __syncthreads();
  if (threadIdx.x == 0) { st->qr_rank[k] = r; st->it[k].prank = -1; st->qr_row[k] = 0; }
}

// The final double-double contraction applies G_k^-1 through a double-double
// LU factorization with partial pivoting of G_k itself, taken from its exact
// FP64 entries: P G_k = L U by Gaussian elimination, the pivot the largest
// leading part in its column (ties to the lowest row), L unit lower triangular
// below the diagonal and U on and above it, hi parts in luh and lo parts in
// lul, column-major with leading dimension cap; lup[k][i] is the row of G_k
// that row i of P G_k holds.  One CTA per interface.  The FP64 QR factors of
// the search carry an error of order u cond(G_k) that no arithmetic after them
// could remove, so they are not used for it.  (The template's FP64 form
// factors in shared memory; the library uses the double-double form.)
template <bool DDM>
__device__ void lu_factor(const Dev &D, State *st, int k, double *As) {
  __shared__ int piv_s;
  const int r = st->r[k], tid = threadIdx.x, nt = blockDim.x, lane = lane_id(), warp = warp_id();
  const int ld = DDM ? D.cap : r;
  double *Ah = DDM ? D.luh[k] : As, *Al = D.lul[k];
  int *perm = D.lup[k];
  for (int e = tid; e < r * r; e += nt) {
    const int a = e % r, b = e / r;
    Ah[a + (size_t)b * ld] = D.Y[k][core_at(D, k, D.lpar[k][a], D.lnode[k][a], b)];
    if (DDM) Al[a + (size_t)b * ld] = 0.0;
  }
  for (int i = tid; i < r; i += nt) perm[i] = i;
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (warp == 0) {                             // pivot row: largest |hi| in column j at or below the diagonal
      double bv = -1.0;
      int bi = 0x7fffffff;
      for (int i = j + lane; i < r; i += 32) {
        const double v = fabs(Ah[i + (size_t)j * ld]);
        if (v > bv) { bv = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (lane == 0) {
        piv_s = bi;
        if (!(bv > 0.0)) st->singular = 1;
      }
    }
    __syncthreads();
    const int pr = piv_s;
    if (pr != j) {                               // swap rows j and pr
      for (int c = tid; c < r; c += nt) {
        const size_t oj = j + (size_t)c * ld, op = pr + (size_t)c * ld;
        const double th = Ah[oj];
        Ah[oj] = Ah[op];
        Ah[op] = th;
        if (DDM) { const double tl = Al[oj]; Al[oj] = Al[op]; Al[op] = tl; }
      }
      if (tid == 0) { const int t = perm[j]; perm[j] = perm[pr]; perm[pr] = t; }
    }
    __syncthreads();
    const double uh = Ah[j + (size_t)j * ld];
    const double ul = DDM ? Al[j + (size_t)j * ld] : 0.0;
    if (uh != 0.0)
      for (int i = j + 1 + tid; i < r; i += nt) {
        const size_t o = i + (size_t)j * ld;
        if (DDM) {
          const dd l = dd_div({Ah[o], Al[o]}, {uh, ul});
          Ah[o] = l.hi; Al[o] = l.lo;
        } else {
          Ah[o] = Ah[o] / uh;
        }
      }
    __syncthreads();
    const int m = r - j - 1;
    if (uh != 0.0)
      for (int e = tid; e < m * m; e += nt) {    // trailing block: a_ic -= l_ij u_jc
        const int i = j + 1 + e % m, c = j + 1 + e / m;
        const size_t oi = i + (size_t)j * ld, oj = j + (size_t)c * ld, o = i + (size_t)c * ld;
        if (DDM) {
          const dd v = dd_add({Ah[o], Al[o]}, dd_neg(dd_mul({Ah[oi], Al[oi]}, {Ah[oj], Al[oj]})));
          Ah[o] = v.hi; Al[o] = v.lo;
        } else {
          Ah[o] = fma(-Ah[oi], Ah[oj], Ah[o]);
        }
      }
    __syncthreads();
  }
  if (!DDM)                                      // the factors to luh, leading dimension cap
    for (int e = tid; e < r * r; e += nt) {
      const int a = e % r, b = e / r;
      D.luh[k][a + (size_t)b * D.cap] = As[a + (size_t)b * r];
    }
  if (tid == 0) atomicAdd(&st->flops[2], (unsigned long long)((DDM ? 20.0 : 2.0) / 3.0 * r * (double)r * r));
}

// the final double-double contraction's factors (double-double runs only)
__global__ void __launch_bounds__(256) k_dd_factor(Dev *const *Dps) {
  __shared__ Dev sD;
  const Dev &D = stage_dev(Dps, sD);
  State *st = D.st;
  const int k = blockIdx.x + 1;
  if (k > D.d - 1 || !D.prec || st->nonfinite || st->singular) return;
  lu_factor<true>(D, st, k, nullptr);
}

// Kernel (c): contraction of the weighted cores with the inverse cross matrices
// (Sec. 4.1), V_1 G_1^-1 V_2 ... G_{d-1}^-1 V_d, as two chains that meet at
// m = (d+1)/2: CTA 0 forms the row x = V_1 G_1^-1 V_2 ... V_m from the left
// (x <- x G_k^-1 = (Q R^-T x^T)^T, then x <- x V_{k+1}), CTA 1 the column
// y = G_m^-1 V_{m+1} ... G_{d-1}^-1 V_d from the right (y <- V_k R^-1 Q^T y),
// and the CTA that finishes second takes the product x y.  R_k is staged in
// shared memory for the sequential substitutions (one warp); the products with
// Q_k and V_k are spread over the threads.  The per-sweep FP64 contraction
// only feeds the stopping rule, so it runs beside the pivot search; a rule
// that fires is recorded as pending and applied at the end of the sweep.
// final_dd: the double-double contraction of the final sets (after the run).

// x <- x G_k^-1 for the row x.  FP64: through the QR factors (R^T t = x,
// x <- Q t).  Double-double (the final contraction, hi/lo pairs): through the
// double-double LU, P G = L U, so x G^-1 = ((x U^-1) L^-1) P.
__device__ void contract_left_solve(const Dev &D, int k, int r, bool prec, double *Rs, double *xh, double *xl,
                                    double *th, double *tl) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = lane_id(), warp = warp_id(), ld = D.cap;
  if (prec) {
    const double *Uh = D.luh[k], *Ul = D.lul[k];
    if (warp == 0) {
      // t U = x: t_j = x_j / U_jj, then x_c -= t_j U_jc for c > j
      for (int j = 0; j < r; ++j) {
        const size_t dj = j + (size_t)j * ld;
        const dd tj = dd_div({xh[j], xl[j]}, {Uh[dj], Ul[dj]});
        for (int c = j + 1 + lane; c < r; c += 32) {
          const size_t o = j + (size_t)c * ld;
          const dd v = dd_add({xh[c], xl[c]}, dd_neg(dd_mul(tj, {Uh[o], Ul[o]})));
          xh[c] = v.hi; xl[c] = v.lo;
        }
        if (lane == 0) { th[j] = tj.hi; tl[j] = tj.lo; }
        __syncwarp();
      }
      // w L = t (unit lower): w_j = t_j, then t_c -= w_j L_jc for c < j, j descending
      for (int j = r - 1; j >= 0; --j) {
        const dd wj = {th[j], tl[j]};
        for (int c = lane; c < j; c += 32) {
          const size_t o = j + (size_t)c * ld;
          const dd v = dd_add({th[c], tl[c]}, dd_neg(dd_mul(wj, {Uh[o], Ul[o]})));
          th[c] = v.hi; tl[c] = v.lo;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = tid; i < r; i += nt) {          // x = w P: x[perm[i]] = w_i
      const int c = D.lup[k][i];
      xh[c] = th[i]; xl[c] = tl[i];
    }
    __syncthreads();
    return;
  }
  // FP64: D^-1 R (row-major), the scaled forward substitution R^T t = x
  stage_compact(Rs, D.Sr[k], nullptr, nullptr, r, ld);
  __syncthreads();
  if (warp == 0) warp_fwd_subst(Rs, xh, th, r, r);
  __syncthreads();
  for (int i = tid; i < r; i += nt) th[i] *= D.rinv[k][i];
  __syncthreads();
  for (int i = tid; i < r; i += nt) {            // x <- Q t
    const double *Qrow = D.Qr[k] + (size_t)i * ld;
    double acc = 0.0;
    for (int j = 0; j < r; ++j) acc = fma(Qrow[j], th[j], acc);
    xh[i] = acc;
  }
  __syncthreads();
}

// y <- G_k^-1 y for the column y.  FP64: through the QR factors (t = Q^T y,
// R z = t).  Double-double (the final contraction): through the double-double
// LU, G^-1 y = U^-1 (L^-1 (P y)).
__device__ void contract_right_solve(const Dev &D, int k, int r, bool prec, double *Rs, double *yh, double *yl,
                                     double *th, double *tl) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = lane_id(), warp = warp_id(), ld = D.cap;
  if (prec) {
    const double *Uh = D.luh[k], *Ul = D.lul[k];
    for (int i = tid; i < r; i += nt) {          // w = P y
      const int c = D.lup[k][i];
      th[i] = yh[c]; tl[i] = yl[c];
    }
    __syncthreads();
    if (warp == 0) {
      // L v = w (unit lower): v_i = w_i, then w_m -= L_mi v_i for m > i
      for (int i = 0; i < r; ++i) {
        const dd vi = {th[i], tl[i]};
        for (int m = i + 1 + lane; m < r; m += 32) {
          const size_t o = m + (size_t)i * ld;
          const dd v = dd_add({th[m], tl[m]}, dd_neg(dd_mul(vi, {Uh[o], Ul[o]})));
          th[m] = v.hi; tl[m] = v.lo;
        }
        __syncwarp();
      }
      // U z = v: z_j = v_j / U_jj, then v_m -= U_mj z_j for m < j, j descending
      for (int j = r - 1; j >= 0; --j) {
        const size_t dj = j + (size_t)j * ld;
        const dd zj = dd_div({th[j], tl[j]}, {Uh[dj], Ul[dj]});
        for (int m = lane; m < j; m += 32) {
          const size_t o = m + (size_t)j * ld;
          const dd v = dd_add({th[m], tl[m]}, dd_neg(dd_mul(zj, {Uh[o], Ul[o]})));
          th[m] = v.hi; tl[m] = v.lo;
        }
        if (lane == 0) { yh[j] = zj.hi; yl[j] = zj.lo; }
        __syncwarp();
      }
    }
    __syncthreads();
    return;
  }
  // FP64: R D^-1 (column-major), the scaled back substitution
  stage_compact(Rs, D.Cc[k], nullptr, nullptr, r, ld);
  for (int i = tid; i < r; i += nt) {            // t = Q^T y
    double acc = 0.0;
    for (int j = 0; j < r; ++j) acc = fma(D.Qr[k][(size_t)j * ld + i], yh[j], acc);
    th[i] = acc;
  }
  __syncthreads();
  if (warp == 0) warp_back_subst(Rs, th, yh, r, r);   // R z = t
  __syncthreads();
  for (int j = tid; j < r; j += nt) yh[j] *= D.rinv[k][j];
  __syncthreads();
}

// value (as hi/lo), the stopping rules (per sweep) or the final value (final_dd)
__device__ void contract_finish(const Dev &D, State *st, dd v, int final_dd) {
  const int d = D.d;
  if (final_dd) {
    v = dd_mul_d(v, D.constant);
    st->value = v.hi;
    st->value_lo = v.lo;
    return;
  }
  const double val = v.hi * D.constant;          // the per-sweep contraction is FP64
  st->value = val;
  st->value_lo = 0.0;
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

__global__ void __launch_bounds__(256) k_contract(Dev *const *Dps, int final_dd) {
  __shared__ Dev sD;
  const Dev &D = stage_dev(Dps, sD);
  pdl_wait();
  pdl_release();
  State *st = D.st;
  if (st->stop && !final_dd) return;
  if (final_dd && (!D.prec || st->nonfinite || st->singular)) return;
  const bool prec = final_dd != 0;
  extern __shared__ double sm[];
  __shared__ double xh[TTQ_MAXR], xl[TTQ_MAXR], th[TTQ_MAXR], tl[TTQ_MAXR];
  __shared__ int is_last;
  const int tid = threadIdx.x, nt = blockDim.x, d = D.d, m = (d + 1) / 2;
  const bool left = blockIdx.x == 0;
  if (st->nonfinite || st->singular) {
    if (tid == 0 && left) {
      st->pending_status = st->nonfinite ? ST_ERR_NONFINITE : ST_ERR_SINGULAR;
      st->stop_pending = 1;
    }
    return;
  }
  double *Rs = sm;
  if (tid == 0 && left) {
    unsigned long long fl = 0;
    for (int k = 1; k <= d - 1; ++k) {
      unsigned long long r = st->r[k], rn = st->r[k + 1];
      fl += (3 * r * r + 2 * r * rn) * (prec ? 15 : 1);
    }
    atomicAdd(&st->flops[2], fl);
  }
  int len;                                       // length of this chain's vector
  if (left) {
    len = st->r[1];
    for (int b = tid; b < len; b += nt) { xh[b] = D.V[1][b]; xl[b] = D.Vlo[1][b]; }
    __syncthreads();
    for (int k = 1; k <= m - 1; ++k) {
      const int r = st->r[k], rn = st->r[k + 1];
      contract_left_solve(D, k, r, prec, Rs, xh, xl, th, tl);
      for (int b = tid; b < rn; b += nt) {      // x <- x V_{k+1}
        if (!prec) {
          double acc = 0.0;
          for (int a = 0; a < r; ++a) acc = fma(xh[a], D.V[k + 1][(size_t)a * D.capL[k + 1] + b], acc);
          th[b] = acc;
        } else {
          dd acc = {0.0, 0.0};
          for (int a = 0; a < r; ++a) {
            const size_t vi = (size_t)a * D.capL[k + 1] + b;
            acc = dd_add(acc, dd_mul({xh[a], xl[a]}, {D.V[k + 1][vi], D.Vlo[k + 1][vi]}));
          }
          th[b] = acc.hi; tl[b] = acc.lo;
        }
      }
      __syncthreads();
      for (int b = tid; b < rn; b += nt) { xh[b] = th[b]; xl[b] = prec ? tl[b] : 0.0; }
      __syncthreads();
      len = rn;
    }
  } else {
    len = st->r[d - 1];
    for (int a = tid; a < len; a += nt) { xh[a] = D.V[d][a]; xl[a] = D.Vlo[d][a]; }
    __syncthreads();
    for (int k = d - 1; k >= m; --k) {
      const int r = st->r[k];
      contract_right_solve(D, k, r, prec, Rs, xh, xl, th, tl);
      if (k == m) break;
      const int rl = st->r[k - 1];
      for (int a = tid; a < rl; a += nt) {       // y <- V_k y
        const size_t row = (size_t)a * D.capL[k];
        if (!prec) {
          double acc = 0.0;
          for (int b = 0; b < r; ++b) acc = fma(D.V[k][row + b], xh[b], acc);
          th[a] = acc;
        } else {
          dd acc = {0.0, 0.0};
          for (int b = 0; b < r; ++b) acc = dd_add(acc, dd_mul({D.V[k][row + b], D.Vlo[k][row + b]}, {xh[b], xl[b]}));
          th[a] = acc.hi; tl[a] = acc.lo;
        }
      }
      __syncthreads();
      for (int a = tid; a < rl; a += nt) { xh[a] = th[a]; xl[a] = prec ? tl[a] : 0.0; }
      __syncthreads();
      len = rl;
    }
  }
  // publish this chain's vector; the CTA that arrives second forms x y
  double *mine = D.cbuf + (left ? 0 : 2 * D.cap);
  for (int a = tid; a < len; a += nt) { mine[a] = xh[a]; mine[D.cap + a] = xl[a]; }
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(&st->contract_arrive, 1u) == 1u);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if (tid == 0) {
    st->contract_arrive = 0;
    const double *other = D.cbuf + (left ? 2 * D.cap : 0);
    dd acc = {0.0, 0.0};
    for (int a = 0; a < len; ++a) {
      const dd o = {__ldcg(other + a), __ldcg(other + D.cap + a)};
      const dd me = {xh[a], xl[a]};
      // the same order in either CTA: x_a y_a summed over a
      acc = prec ? dd_add(acc, dd_mul(left ? me : o, left ? o : me)) : dd{fma(me.hi, o.hi, acc.hi), 0.0};
    }
    contract_finish(D, st, acc, final_dd);
  }
}

// Pass 2 of the argmax of a search stage (whole CTA, interface k): the first
// candidate index whose score lies in the tie window below the stage maximum,
// -1 if the stage had no eligible candidate.  Clears the stage reduction.
//   stage 0 (samples): a scan of the S sample scores.
//   stage 1 (column step, rho = alpha N_k + i): slot w = alpha rows + q holds the
//     maximum over the 32 nodes i of row q, so the answer lies in the first slot
//     whose maximum reaches the window; one scan of its 32 candidates.
//   stage 2 (row step, gamma = j r_{k+1} + beta): slot w = beta rows + q holds the
//     maximum over the nodes j of row q of fiber beta; the answer has the smallest
//     j, so it lies in the lowest row any qualifying slot reaches; the qualifying
//     slots of that row are scanned.
// The first loads (the stage maximum and count, the scale, the outer rank, the
// item rows and the first 4 blockDim candidates, read up to the arrays'
// capacity before their counts are known) form one round, so a pick costs two
// dependent rounds of global reads.  qbits: blockDim.x words of shared scratch
// (stage 2 marks the qualifying items there, TTQ_MAXR * TTQ_MAX_NODES / 32 bits
// at most).  vrow (stage 1, may be null): L_k(rho*, :) (r entries) is read into
// it by the warp that finds rho*, before the block learns the result, and with
// it, into fm, the node indices of rho*'s modes 0 .. k-1 (the next row step's
// fixed modes), in the same round of loads.
__device__ int stage_pick(const Dev &D, int k, int j, int stage, double *e_out, unsigned *qbits,
                          double *vrow = nullptr, int r = 0, int *fm = nullptr) {
  __shared__ int si[TTQ_WARPS];
  __shared__ double se[TTQ_WARPS];
  State *st = D.st;
  IfaceState &I = search_state(D, st, k, j);
  const int tid = threadIdx.x, nt = blockDim.x, lane = lane_id(), warp = warp_id(), nw = nt >> 5;
  const long long *csb = reinterpret_cast<const long long *>(cs_of(D, k, j));
  const double *ce = ce_of(D, k, j);
  const long long *imb = reinterpret_cast<const long long *>(im_of(D, k, j));
  const long long *src = stage == 0 ? csb : imb;
  const int Nm = stage == 1 ? D.N[k - 1] : D.N[k];           // nodes of the searched mode
  const int lim = stage == 0 ? D.S[k] : D.cap * ((Nm + 31) >> 5);
  const unsigned long long mbits = __ldcg(&I.smax_bits);
  const unsigned n = __ldcg(&I.stage_count);
  const double scale = __longlong_as_double((long long)__ldcg(&st->scale_bits));
  const int rm = stage == 0 ? 0 : __ldcg(stage == 1 ? &st->r[k - 1] : &st->r[k + 1]);
  long long vb[4];
  double ev[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int t = tid + u * nt;
    vb[u] = t < lim ? __ldcg(src + t) : -1LL;
    ev[u] = (stage == 0 && t < lim) ? __ldcg(ce + t) : 0.0;
  }
  if (stage == 2) qbits[tid] = 0u;
  __syncthreads();                               // all have read the reduction before it is cleared
  if (tid == 0) { I.smax_bits = 0ULL; I.stage_count = 0; }
  if (n == 0) { *e_out = 0.0; return -1; }
  const double smax = __longlong_as_double((long long)mbits);
  const double thr = __dadd_rn(smax, -__dadd_rn(__dmul_rn(TTQ_TIE_REL, smax), __dmul_rn(TTQ_TIE_ABS, scale)));
  // a score qualifies if it is eligible (>= 0) and within the window (>= thr):
  // scores are non-negative doubles or -1, so this is one signed comparison of
  // bit patterns (integer pipe, not the FP64 unit)
  const long long thrb = thr > 0.0 ? __double_as_longlong(thr) : 0LL;
  if (stage == 0) {
    const int Sk = lim;
    int first = 0x7fffffff;
    double efirst = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = tid + u * nt;
      if (t < Sk && vb[u] >= thrb && t < first) { first = t; efirst = ev[u]; }
    }
    for (int t0 = tid + 4 * nt; t0 < Sk; t0 += 4 * nt) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {           // four candidates' loads in flight
        const int t = t0 + u * nt;
        vb[u] = t < Sk ? __ldcg(csb + t) : -1LL;
        ev[u] = t < Sk ? __ldcg(ce + t) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = t0 + u * nt;
        if (vb[u] >= thrb && t < first) { first = t; efirst = ev[u]; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int ov = __shfl_xor_sync(0xffffffffu, first, o);
      const double oe = __shfl_xor_sync(0xffffffffu, efirst, o);
      if (ov < first) { first = ov; efirst = oe; }
    }
    if (lane == 0) { si[warp] = first; se[warp] = efirst; }
    __syncthreads();
    first = si[0];
    efirst = se[0];
    for (int w = 1; w < nw; ++w)
      if (si[w] < first) { first = si[w]; efirst = se[w]; }
    *e_out = efirst;
    return first;                                // n > 0: some score reaches the window
  }
  const NodeChunks nc = node_chunks(Nm, 1);      // a slot per row of 32 nodes
  const int nch = nc.nch;
  int wmin = 0x7fffffff;                       // first qualifying slot (stage 1) / its chunk (stage 2)
  const int nslot = rm * nch;
  for (int w0 = tid; w0 < nslot; w0 += 4 * nt) {
    if (w0 != tid) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {            // four slots' loads in flight
        const int w = w0 + u * nt;
        vb[u] = w < nslot ? __ldcg(imb + w) : -1LL;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int w = w0 + u * nt;
      if (w < nslot && vb[u] >= thrb) {
        wmin = min(wmin, stage == 1 ? w : w % nch);
        if (stage == 2) atomicOr(qbits + (w >> 5), 1u << (w & 31));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wmin = min(wmin, __shfl_xor_sync(0xffffffffu, wmin, o));
  if (lane == 0) si[warp] = wmin;
  __syncthreads();
  wmin = si[0];
  for (int w = 1; w < nw; ++w) wmin = min(wmin, si[w]);
  __syncthreads();                               // si is reused below
  int f = 0x7fffffff;
  double fe = 0.0;
  if (stage == 1) {
    if (warp == 0) {
      const int alpha = wmin / nch, ch = wmin % nch;
      int i0, i1, nq;
      chunk_span(nc, ch, Nm, i0, i1, nq);
#pragma unroll
      for (int q = 0; q < TTQ_CHUNK / 32; ++q) {
        const int i = i0 + lane + 32 * q;
        if (i < i1) {
          const int c = alpha * Nm + i;
          const long long v = __ldcg(csb + c);
          const double e = __ldcg(ce + c);
          if (v >= thrb && c < f) { f = c; fe = e; }
        }
      }
      if (vrow) {                                // stage 1's answer is this warp's
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const int of = __shfl_xor_sync(0xffffffffu, f, o);
          const double oe = __shfl_xor_sync(0xffffffffu, fe, o);
          if (of < f) { f = of; fe = oe; }
        }
        if (f != 0x7fffffff) {
          const int ai = f / Nm, ii = f % Nm;
          const int fmv = lane < k - 1 ? D.lidx[k - 1][ai * D.d + lane] : ii;
          for (int b = lane; b < r; b += 32) vrow[b] = D.Y[k][core_at(D, k, ai, ii, b)];
          if (fm && lane < k) fm[lane] = fmv;
        }
      }
    }
  } else {
    // the qualifying items of chunk ch, a warp each (their marks are in shared memory)
    const int ch = wmin;
    int j0, j1, nq;
    chunk_span(nc, ch, Nm, j0, j1, nq);
    for (int beta = warp; beta < rm; beta += nw) {
      const int w = beta * nch + ch;
      if (!((qbits[w >> 5] >> (w & 31)) & 1u)) continue;
#pragma unroll
      for (int q = 0; q < TTQ_CHUNK / 32; ++q) {
        const int j = j0 + lane + 32 * q;
        if (j < j1) {
          const int c = j * rm + beta;
          const long long v = __ldcg(csb + c);
          const double e = __ldcg(ce + c);
          if (v >= thrb && c < f) { f = c; fe = e; }
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int of = __shfl_xor_sync(0xffffffffu, f, o);
    const double oe = __shfl_xor_sync(0xffffffffu, fe, o);
    if (of < f) { f = of; fe = oe; }
  }
  if (lane == 0) { si[warp] = f; se[warp] = fe; }
  __syncthreads();
  f = si[0];
  fe = se[0];
  for (int w = 1; w < nw; ++w)
    if (si[w] < f) { f = si[w]; fe = se[w]; }
  *e_out = fe;
  return f;
}

// Scratch of the decisions between search stages (one CTA)
struct SolveSmem {
  double v[TTQ_MAXR], t[TTQ_MAXR], ri[TTQ_MAXR], part[4 * TTQ_MAXR];
  int is_last;
};

// Whether interface k's rook steps take their shared pair factors from the
// step's table: the R^n form of D on one uniform grid, from rank 24 on (below,
// the solve's substitution is too short to hide building it and the rook items
// are latency bound).  The solve and the rook kernels decide alike.
__device__ __forceinline__ bool uses_ptab(const Dev &D, int rk) {
  return D.family == FAM_D && D.form == FORM_RN && D.uniformT && rk >= 24;
}

// The next rook step's pair factors that every fiber of the step shares (R^n
// form of D on one uniform grid): a column step (free mode k-1) shares the
// modes k.. of gamma* = (j, beta), a row step (free mode k) the modes ..k-1 of
// rho* = (alpha, i).  Built by warps 1.. of the CTA while warp 0 runs the
// substitution; fm: the fixed node indices of those modes (shared memory).
__device__ __forceinline__ void build_ptab(const Dev &D, int k, int j, bool col, const int *fm, int nfm) {
  // only warps on the other three schedulers (warp w runs on scheduler w % 4),
  // so the FP64 unit of warp 0's substitution chain is not shared
  const int w = warp_id(), nw = blockDim.x >> 5;
  if ((w & 3) == 0) return;
  const int slot = (w - 1 - w / 4) * 32 + lane_id();            // 0 .. (3/4 nw - 1) * 32 + 31
  const int nslots = (nw - (nw + 3) / 4) * 32;
  const int Nf = col ? D.N[k - 1] : D.N[k];
  double *tab = ptab_of(D, k, j);
  for (int i = slot; i < Nf; i += nslots) {
    double p = 1.0;
    for (int q = 0; q < nfm; ++q) {
      const int dm = i - fm[q];
      p *= D.T[dm < 0 ? -dm : dm];
    }
    tab[i] = p;
  }
}

// Decisions of Alg. 2 after a search stage for interface k, by one CTA after the
// stage's last work item of k: the argmax of the stage (pass 2),
// the interface's search state, and the solve the next stage needs.
//   mode 0, after the random samples: (rho*, gamma*) of the best sample; column
//           solve z = G^-1 y, y = R_{k+1}(:, gamma*) = Y_{k+1}(:, j, beta).
//   mode 1, after a column step: rho* = argmax over E(:, gamma*); row solve
//           b = G^-T l, l = L_k(rho*, :)^T = Y_k(alpha, i, :), unless rho* is
//           the previous round's row (the rook test, Eq. 2, then ends the search).
//   mode 2, after a row step: gamma_new = argmax over E(rho*, :); the rook test
//           (Eq. 2) or the round limit ends the search, else the next column solve.
// The solve's result goes to the search's zvec; the row solve of search 0 also
// keeps R^-T l in pvec[k] for the QR update of the pivot's row.  j: the search
// of interface k (0 .. npiv-1); pick_in >= 0 (mode 0): the sample that starts
// it, with residual e_in, instead of the stage's argmax.  Fs: the scaled triangle the solve needs
// (R D^-1 column-major for modes 0 and 2, D^-1 R row-major for mode 1) and Qs
// (Q row-major / column-major), both compact with leading dimension r, when the
// caller has them in shared memory; nullptr reads them from global memory.
// ri: 1/R_jj in shared memory, or nullptr.
__device__ void stage_finish(const Dev &D, int k, int j, int mode, const double *Fs, const double *Qs,
                             const double *ri_s, SolveSmem &sc, bool staging_in_flight = false, int pick_in = -1,
                             double e_in = 0.0) {
  State *st = D.st;
  IfaceState &I = search_state(D, st, k, j);
  double *zv = zvec_of(D, k, j);
  const int r = st->r[k], ld = D.cap, tid = threadIdx.x, nt = blockDim.x;
  double *v = sc.v, *t = sc.t;
  const double *ri = ri_s;
  if (!ri) {
    for (int b = tid; b < r; b += nt) sc.ri[b] = D.rinv[k][b];
    ri = sc.ri;
  }
  const double *F = Fs ? Fs : (mode == 1 ? D.Sr[k] : D.Cc[k]);
  const int fld = Fs ? r : ld;
  unsigned *qb = reinterpret_cast<unsigned *>(sc.part);   // free until the solve's products
  __shared__ int fm[TTQ_MAXD];
  double e;
  int col = -1, row = -1, spick = -1;
  // the search state the rook test reads, loaded with the argmax's first round
  // (nothing writes it before the argmax's barriers)
  const int prev_row = mode == 1 ? __ldcg(&I.row) : 0, prev_col = mode == 2 ? __ldcg(&I.col) : 0;
  const int done_rounds = mode != 0 ? __ldcg(&I.rounds) : 0;
  if (mode == 0) {
    int pick = pick_in;
    if (pick_in >= 0) e = e_in;
    else pick = stage_pick(D, k, j, 0, &e, qb);
    spick = pick;
    if (pick >= 0) {
      const int Nk = D.N[k - 1], Nk1 = D.N[k], rn = st->r[k + 1];
      const unsigned long long sid = stream_id(st->sweep, k, 1);
      row = draw_index(D.seed, sid, 2ULL * pick, (unsigned long long)st->r[k - 1] * Nk);
      col = draw_index(D.seed, sid, 2ULL * pick + 1, (unsigned long long)Nk1 * rn);
      if (tid == 0) { I.row = row; I.col = col; I.err = e; I.active = 1; }
    }
  } else if (mode == 1) {
    const int pick = stage_pick(D, k, j, 1, &e, qb, v, r, fm);   // L_k(rho*, :) lands in v, its modes in fm
    const int prev = prev_row;
    // Eq. 2 already holds when the column search returns the row searched in the
    // previous round: that search returned the current column, so the pivot
    // dominates its row and its column and the search ends without a row search
    const bool rook = pick >= 0 && done_rounds >= 1 && pick == prev;
    if (tid == 0) {
      if (pick < 0) I.active = 0;
      else if (rook) { I.rounds = done_rounds + 1; I.rook_done = 1; }
      else I.row = pick;
    }
    row = rook ? -1 : pick;
  } else {
    const int pick = stage_pick(D, k, j, 2, &e, qb);
    if (pick < 0) {
      if (tid == 0) I.active = 0;
    } else {
      const int rounds = done_rounds + 1;
      const bool done = (pick == prev_col) || rounds >= D.rook_max;
      if (tid == 0) { I.rounds = rounds; I.col = pick; I.err = e; I.rook_done = done ? 1 : 0; }
      if (!done) col = pick;
    }
  }
  const bool colsolve = mode != 1 && col >= 0, rowsolve = mode == 1 && row >= 0;
  const bool tab = uses_ptab(D, r) && (colsolve || rowsolve) && blockDim.x > 32;
  int nfm = 0;
  // the node indices the next rook step fixes go to I.fix, so that its work
  // items read them in their first round of loads
  if (colsolve) {
    const int rn = st->r[k + 1], j = col / rn, beta = col % rn;
    if (mode != 0)                               // after the samples the best sample's z is at hand
      for (int b = tid; b < r; b += nt) v[b] = D.Y[k + 1][core_at(D, k + 1, b, j, beta)];
    nfm = D.d - k;                               // modes k .. d-1
    if (tid < nfm) {
      fm[tid] = tid == 0 ? j : D.ridx[k + 1][beta * D.d + k + tid];
      I.fix[k + tid] = fm[tid];
    }
  } else if (rowsolve) {
    nfm = k;                                     // modes 0 .. k-1, read with L_k(rho*, :) by the argmax
    if (tid < nfm) I.fix[tid] = fm[tid];
  }
  if (staging_in_flight) cp_async_wait_all();   // factors copied under the argmax
  __syncthreads();
  if (colsolve && mode == 0) {
    for (int b = tid; b < r; b += nt) zv[b] = __ldcg(D.zs[k] + (size_t)spick * D.cap + b);
    if (tab) build_ptab(D, k, j, true, fm, nfm);
  } else if (colsolve) {
    // t = Q^T y (Q row-major: Q[b][i] at Q[b ld + i]), then R z = t
    if (Qs) cta_gemv(Qs, 1, r, v, r, sc.part, t);
    else cta_gemv(D.Qr[k], 1, ld, v, r, sc.part, t);
    if (warp_id() == 0) warp_back_subst(F, t, v, r, fld);
    else if (tab) build_ptab(D, k, j, true, fm, nfm);
    __syncthreads();
    for (int b = tid; b < r; b += nt) zv[b] = v[b] * ri[b];
  } else if (rowsolve) {
    // R^T t = l, then b = Q t (Q column-major: Q[i][c] at Q[i + c ld])
    if (warp_id() == 0) warp_fwd_subst(F, v, t, r, fld);
    else if (tab) build_ptab(D, k, j, false, fm, nfm);
    __syncthreads();
    for (int b = tid; b < r; b += nt) t[b] *= ri[b];
    __syncthreads();
    if (Qs) cta_gemv(Qs, 1, r, t, r, sc.part, v);
    else cta_gemv(D.Qc[k], 1, ld, t, r, sc.part, v);
    for (int b = tid; b < r; b += nt) {
      zv[b] = v[b];
      if (j == 0) D.pvec[k][b] = t[b];
    }
    if (tid == 0 && j == 0) { I.prow = row; I.prank = r; }
  }
  if (((colsolve && mode != 0) || rowsolve) && tid == 0)
    atomicAdd(&st->flops[9], (unsigned long long)(3 * r * r) +
                                 (tab ? (unsigned long long)(colsolve ? D.N[k - 1] : D.N[k]) * nfm : 0ULL));
  __syncthreads();
}

// End of the sweep (Alg. 6), in the last decisions kernel of the search: every
// CTA appends its interface's accepted pivot (new row alpha* + i* of I<=k, new
// column j* + beta* of I>k, nested by construction; the neighbours' sets are
// read below their current ranks, which no CTA changes before all have
// arrived), then the last CTA of the instance to arrive applies the ranks, the
// stopping rules and the sweep count and, inside the whole-run graph, sets the
// WHILE condition: continue while the run is not over, never past max_sweeps.
// The accepted pivot of interface k appended to its nested sets (warp 0 of
// the calling CTA): new row alpha* + i* of I<=k, new column j* + beta* of
// I>k, nested by construction; the neighbours' sets are read below their
// current ranks, which nothing changes before the end of the sweep.
__device__ void sweep_append(const Dev &D, State *st, int k) {
  if (warp_id() != 0) return;
  const int d = D.d, lane = lane_id();
  IfaceState &I = st->it[k];
  const double scale = __longlong_as_double((long long)st->scale_bits);
  const int a = st->r[k];
  const int active = __ldcg(&I.active);
  const int prow = __ldcg(&I.row), pcol = __ldcg(&I.col);
  const bool acc = active && fabs(__ldcg(&I.err)) > D.pivot_tol * scale && a < D.cap;
  if (lane == 0 && active) I.accepted = acc ? 1 : 0;
  if (acc) {
    const int Nk = D.N[k - 1], rn = st->r[k + 1];
    const int alpha = prow / Nk, i = prow % Nk, j = pcol / rn, beta = pcol % rn;
    if (lane < d) {
      const int m = lane;
      D.lidx[k][(size_t)a * d + m] = (m < k - 1) ? D.lidx[k - 1][alpha * d + m] : (m == k - 1 ? i : -1);
      D.ridx[k][(size_t)a * d + m] = (m == k) ? j : (m > k ? D.ridx[k + 1][beta * d + m] : -1);
    }
    if (lane == 0) {
      D.lpar[k][a] = alpha; D.lnode[k][a] = i;
      D.rpar[k][a] = beta; D.rnode[k][a] = j;
    }
  }
}

// The end of the sweep proper (one whole CTA, after every interface's append
// and the contraction): the ranks of the interfaces that accepted a pivot, the
// sweep's evaluations, the stopping rules and the sweep count; inside the
// whole-run graph it sets the WHILE condition: continue while the run is not
// over, never past max_sweeps.  A search that gave up waiting (its wait limit
// passed) ends the run with status TIMEOUT.
__device__ void sweep_finalize(const Dev &D, State *st, bool append, cudaGraphConditionalHandle h, int use_cond) {
  const int d = D.d, tid = threadIdx.x;
  __shared__ int nacc_s;
  __shared__ unsigned long long ev_s;
  if (tid == 0) { nacc_s = 0; ev_s = 0ULL; }
  __syncthreads();
  if (append) {
    // a thread per interface: its rank, the sweep's evaluations, the accepted count
    for (int q = tid + 1; q <= d - 1; q += blockDim.x) {
      IfaceState &I = st->it[q];
      if (D.npiv > 1) {
        // several pivots per sweep: the count multi_accept kept, every search's evaluations
        unsigned long long ev = 0;
        for (int j = 0; j < D.npiv; ++j) ev += __ldcg(&search_state(D, st, q, j).evals);
        atomicAdd(&ev_s, ev);
        const int na = __ldcg(&I.accepted);
        if (na > 0) {
          st->r[q] += na;
          atomicAdd(&nacc_s, 1);
        }
      } else {
        atomicAdd(&ev_s, I.evals);
        if (I.active && I.accepted) {
          st->r[q] += 1;
          atomicAdd(&nacc_s, 1);
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    st->end_arrive = 0;
    if (st->stop) {
    } else if (st->search_abort) {
      st->stop = 1;
      st->status = ST_ERR_TIMEOUT;
    } else if (st->stop_pending) {
      st->stop = 1;
      st->status = st->pending_status;
    } else if (!st->search) {
      st->sweep++;
    } else {
      st->search_evals += (long long)ev_s;
      if (st->rules && nacc_s == 0) { st->stop = 1; st->status = ST_NO_PIVOT; }
      st->sweep++;
    }
    if (use_cond) {
      const int guard = ++st->loop_guard;
      const int cont = !st->stop && st->sweep < D.max_sweeps && guard < D.max_sweeps + 2;
      cudaGraphSetConditional(h, cont ? 1u : 0u);
    }
  }
}

// Several pivots per interface per sweep (a rank-adaptive variant; Alg. 6
// adds one): interface k's pivots from the rook searches of its npiv starts,
// by the last CTA of its searches in the sweep's last decisions kernel (whole
// CTA).  On the residual E of the sweep's old cross:
//   1. searches that found a pivot, in start order; one whose row or column
//      equals that of an earlier kept search is dropped;
//   2. M(a, c) = E(x_a, y_c) over the kept rows x_a and columns y_c: M(a, a)
//      is search a's residual, the others A(x_a, y_c) - L_k(x_a, :) z_c, z_c =
//      G_k^-1 R_{k+1}(:, y_c) (a warp each: Q^T y, back substitution) and A
//      evaluated at the points (groups of 8 lanes);
//   3. greedy complete pivoting: the largest |M| over the rows and columns
//      left (tie window, first in row-major order) while it exceeds
//      pivot_tol * scale and the rank stays below the cap; its row and column
//      are appended (nested by construction, as sweep_append) and M becomes
//      its Schur complement M_be - M_bc M_ae / M_ac.
// The count kept goes to it[k].accepted.
__device__ void multi_accept(const Dev &D, State *st, int k, bool append) {
  __shared__ int kr[TTQ_MAXP], kc[TTQ_MAXP], km_s, acc_a[TTQ_MAXP], acc_c[TTQ_MAXP], nacc_s;
  __shared__ double ke[TTQ_MAXP], Mx[TTQ_MAXP][TTQ_MAXP], Av[TTQ_MAXP][TTQ_MAXP];
  __shared__ double zc[TTQ_MAXP][TTQ_MAXR], tv[TTQ_MAXP][TTQ_MAXR], yv[TTQ_MAXP][TTQ_MAXR];
  __shared__ int mxp[TTQ_MAXD][TTQ_MAXP * TTQ_MAXP];   // node indices of point q = a m + c in column q
  const int tid = threadIdx.x, lane = lane_id(), warp = warp_id(), nw = blockDim.x >> 5, d = D.d;
  IfaceState &I0 = st->it[k];
  if (!append) {
    if (tid == 0) I0.accepted = 0;
    return;
  }
  const int r = st->r[k], ld = D.cap, Nk = D.N[k - 1], rn = st->r[k + 1];
  const double scale = __longlong_as_double((long long)__ldcg(&st->scale_bits));
  if (tid == 0) {
    int m = 0;
    for (int j = 0; j < D.npiv; ++j) {
      IfaceState &I = search_state(D, st, k, j);
      if (!__ldcg(&I.active) || __ldcg(&I.merged)) continue;
      const int rw = __ldcg(&I.row), cl = __ldcg(&I.col);
      bool dup = false;
      for (int q = 0; q < m; ++q) dup |= (kr[q] == rw) || (kc[q] == cl);
      if (dup) continue;
      kr[m] = rw;
      kc[m] = cl;
      ke[m] = __ldcg(&I.err);
      ++m;
    }
    km_s = m;
  }
  __syncthreads();
  const int m = km_s;
  if (m >= 2) {
    // z_c = G^-1 R_{k+1}(:, y_c): t = Q^T y (Q row-major), R D^-1 back substitution, D^-1
    if (warp < m) {
      const int jc = kc[warp] / rn, bc = kc[warp] % rn;
      for (int b = lane; b < r; b += 32) yv[warp][b] = D.Y[k + 1][core_at(D, k + 1, b, jc, bc)];
      __syncwarp();
      for (int i = lane; i < r; i += 32) {
        double acc = 0.0;
        for (int b = 0; b < r; ++b) acc = fma(D.Qr[k][(size_t)b * ld + i], yv[warp][b], acc);
        tv[warp][i] = acc;
      }
      __syncwarp();
      warp_back_subst(D.Cc[k], tv[warp], zc[warp], r, ld);
      __syncwarp();
      for (int b = lane; b < r; b += 32) zc[warp][b] *= D.rinv[k][b];
    }
    // the points (x_a, y_c): modes ..k-2 from I<=k-1, i_a, j_c, modes k+1.. from I>k+1
    const int mm = m * m;
    for (int e = tid; e < d * mm; e += blockDim.x) {
      const int v = e / mm, q = e % mm, a = q / m, c = q % m;
      const int alpha = kr[a] / Nk, i = kr[a] % Nk, jj = kc[c] / rn, beta = kc[c] % rn;
      int mv;
      if (v < k - 1) mv = D.lidx[k - 1][alpha * d + v];
      else if (v == k - 1) mv = i;
      else if (v == k) mv = jj;
      else mv = D.ridx[k + 1][beta * d + v];
      mxp[v][q] = mv;
    }
    __syncthreads();
    if (warp < (mm + 3) / 4) {                   // four points per warp, a group of 8 lanes each
      const int g = lane >> 3, gl = lane & 7, q = warp * 4 + g;
      const double A = group_point_value<8>(D, &mxp[0][q < mm ? q : 0], TTQ_MAXP * TTQ_MAXP, gl);
      if (gl == 0 && q < mm) Av[q / m][q % m] = A;
    }
    __syncthreads();
    for (int q = warp; q < mm; q += nw) {
      const int a = q / m, c = q % m;
      if (a == c) continue;
      const int alpha = kr[a] / Nk, i = kr[a] % Nk;
      double acc = 0.0;
      for (int b = lane; b < r; b += 32) acc = fma(D.Y[k][core_at(D, k, alpha, i, b)], zc[c][b], acc);
      acc = warp_sum(acc);
      if (lane == 0) Mx[a][c] = Av[a][c] - acc;
    }
  }
  if (tid < m) Mx[tid][tid] = ke[tid];
  __syncthreads();
  if (tid == 0) {
    unsigned rows_left = (1u << m) - 1u, cols_left = (1u << m) - 1u;
    int n = 0;
    while (rows_left && n < D.cap - r) {
      double smax = -1.0;
      for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c)
          if (((rows_left >> a) & 1u) && ((cols_left >> c) & 1u) && isfinite(Mx[a][c])) smax = fmax(smax, fabs(Mx[a][c]));
      if (smax < 0.0) break;
      const double thr = __dadd_rn(smax, -__dadd_rn(__dmul_rn(TTQ_TIE_REL, smax), __dmul_rn(TTQ_TIE_ABS, scale)));
      int fa = -1, fc = -1;
      for (int a = 0; a < m && fa < 0; ++a)
        for (int c = 0; c < m; ++c)
          if (((rows_left >> a) & 1u) && ((cols_left >> c) & 1u) && isfinite(Mx[a][c]) && fabs(Mx[a][c]) >= thr) {
            fa = a;
            fc = c;
            break;
          }
      const double piv = Mx[fa][fc];
      if (!(fabs(piv) > D.pivot_tol * scale)) break;
      acc_a[n] = fa;
      acc_c[n] = fc;
      ++n;
      rows_left &= ~(1u << fa);
      cols_left &= ~(1u << fc);
      for (int b = 0; b < m; ++b)
        for (int e = 0; e < m; ++e)
          if (((rows_left >> b) & 1u) && ((cols_left >> e) & 1u))
            Mx[b][e] = __dsub_rn(Mx[b][e], __ddiv_rn(__dmul_rn(Mx[b][fc], Mx[fa][e]), piv));
    }
    nacc_s = n;
    I0.accepted = n;
    if (m > 1) atomicAdd(&I0.evals, (unsigned long long)(m * (m - 1)));
  }
  __syncthreads();
  const int n = nacc_s;
  if (warp == 0)
    for (int t = 0; t < n; ++t) {
      const int prow = kr[acc_a[t]], pcol = kc[acc_c[t]], pos = r + t;
      const int alpha = prow / Nk, i = prow % Nk, jj = pcol / rn, beta = pcol % rn;
      if (lane < d) {
        D.lidx[k][(size_t)pos * d + lane] = (lane < k - 1) ? D.lidx[k - 1][alpha * d + lane] : (lane == k - 1 ? i : -1);
        D.ridx[k][(size_t)pos * d + lane] = (lane == k) ? jj : (lane > k ? D.ridx[k + 1][beta * d + lane] : -1);
      }
      if (lane == 0) {
        D.lpar[k][pos] = alpha; D.lnode[k][pos] = i;
        D.rpar[k][pos] = beta; D.rnode[k][pos] = jj;
      }
    }
}

// End of the sweep (Alg. 6) in the last decisions kernel of the staged search:
// every CTA appends its interface's accepted pivot, then the last CTA of the
// instance to arrive finalizes the sweep.
template <bool MULTI>
__device__ void sweep_end(const Dev &D, int k, bool mine, cudaGraphConditionalHandle h, int use_cond) {
  State *st = D.st;
  __shared__ int last_s;
  const bool append = !st->stop && !st->stop_pending && st->search && !st->search_abort;
  if constexpr (MULTI) {
    // one CTA per search of the interface (grid y): the last of them to
    // arrive takes the interface's pivots from all of its searches
    if (mine) {
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) last_s = (atomicAdd(&st->it[k].acc_arrive, 1u) == gridDim.y - 1) ? 1 : 0;
      __syncthreads();
      if (last_s) {
        __threadfence();
        multi_accept(D, st, k, append);
      }
    }
  } else if (append && mine) {
    sweep_append(D, st, k);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_s = (atomicAdd(&st->end_arrive, 1u) == gridDim.x * gridDim.y - 1) ? 1 : 0;
  __syncthreads();
  if (!last_s) return;
  __threadfence();
  sweep_finalize(D, st, append, h, use_cond);
}

// The decisions after a rook step (modes 1 and 2 of stage_finish), one CTA per
// interface and search.  The rank and the factors are fixed from kernel (b) to the end of
// the search, so their copies to shared memory are issued before the wait for
// the preceding rook step: they overlap its tail (the rook step streams the
// cores through L2, so the factors come from DRAM) instead of delaying the argmax.
// fin: the search's last decisions kernel, which also ends the sweep (sweep_end).
// MULTI: several pivots per sweep (one CTA per search, grid y); the one-pivot
// instance is the same code with the search index 0
template <bool MULTI>
__global__ void __launch_bounds__(256) k_solve(Dev *const *Dps, int mode, int fin, cudaGraphConditionalHandle h,
                                               int use_cond) {
  __shared__ Dev sD;
  const Dev &D = stage_dev(Dps, sD);
  State *st = D.st;
  const int k = blockIdx.x + 1, j = MULTI ? (int)blockIdx.y : 0;  // interface, search (grid y: its searches)
  const bool mine = k <= D.d - 1;
  extern __shared__ double sm[];
  __shared__ SolveSmem sc;
  const int r = mine ? st->r[k] : 0, ld = D.cap;
  double *Fs = sm;
  double *Qs = D.q_in_smem ? sm + (size_t)r * r : nullptr;   // Q staged too when it fits
  // the run flags and the search's state were last written two or more
  // launches back (the previous decisions kernel, the samples' finisher, the
  // end of the previous sweep), which had completed before the preceding rook
  // step passed its own wait: they are read before this kernel's wait
  bool work = false;
  if (mine) {
    const IfaceState &I = search_state(D, st, k, j);
    work = !st->stop && st->search && I.active && !I.rook_done;
  }
  if (r > 0 && work) {
    if (mode == 1) stage_compact_async(Fs, D.Sr[k], Qs, D.Qc[k], r, ld);   // D^-1 R row-major, Q col-major
    else stage_compact_async(Fs, D.Cc[k], Qs, D.Qr[k], r, ld);             // R D^-1 col-major, Q row-major
    for (int b = threadIdx.x; b < r; b += blockDim.x) cp_async8(sc.ri + b, D.rinv[k] + b);
  }
  pdl_wait();
  pdl_release();
  // a search that met an earlier one in the preceding rook step stops (set by
  // that step, so read after the wait and through L2)
  if (MULTI && work && __ldcg(&search_state(D, st, k, j).merged)) work = false;
  if (work)
    stage_finish(D, k, j, mode, Fs, Qs, sc.ri, sc, true);
  else
    cp_async_wait_all();                         // no copy outlives the CTA
  if (fin) sweep_end<MULTI>(D, k, mine, h, use_cond);
}

// per-warp scratch of the rook kernels (no solve buffers: the solves run in k_solve)
struct RookSmem {
  int ms[TTQ_WARPS][TTQ_MAXD];
  double pl[TTQ_WARPS][TTQ_MAXPAIR];
  int exc[TTQ_WARPS][TTQ_MAXR];
  __align__(16) double z[TTQ_WARPS][TTQ_MAXR];   // read two entries at a time
};

// a stage's candidates of one warp feed the interface's maximum (pass 1 of the
// argmax; IEEE bits of non-negative doubles order like the values)
__device__ __forceinline__ void stage_publish(IfaceState &I, double best, unsigned nelig) {
  if (nelig) {
    atomicMax(&I.smax_bits, (unsigned long long)__double_as_longlong(best));
    atomicAdd(&I.stage_count, nelig);
  }
}

__device__ __forceinline__ bool iface_searchable(const Dev &D, const State *st, int k) {
  if (k > D.d - 1) return false;            // instances with fewer interfaces (batches)
  if (st->stop || !st->search) return false;
  // sequential sweep: only the step's interface, and none once a stopping rule fired
  if (st->seq_k && (k != st->seq_k || st->stop_pending)) return false;
  const int rk = st->r[k];
  if (rk >= D.cap) return false;
  if (st->r[k - 1] * D.N[k - 1] <= rk) return false;
  if (D.N[k] * st->r[k + 1] <= rk) return false;
  return true;
}

// Alg. 2, first step: residuals E = A - L_k G_k^-1 R_{k+1} at seeded random
// positions (rho_t, gamma_t) of superblock k.  A warp takes TTQ_SPW samples at a
// time: one lane each evaluates A at its point, then a group of TTQ_SG lanes per
// sample forms z = G_k^-1 R_{k+1}(:, gamma_t) = R^-1 (Q^T y) (rows of Q^T y and
// of the back substitution split over the group, so one warp instruction of the
// sequential substitution serves TTQ_SPW samples) and E = A - L_k(rho_t, :) z.
#ifndef TTQ_SG
#define TTQ_SG 8
#endif
#define TTQ_SPW (32 / TTQ_SG)
// One sample's interpolant L_k(rho, :) G_k^-1 y by a group of TTQ_SG lanes, with
// the group's vector in registers: lane gl holds rows gl + TTQ_SG m, m < NB
// (NB = the row blocks of r_k <= TTQ_SG NB).  t = Q^T y is formed for all of a lane's rows in
// one pass over y, the back substitution with R D^-1 takes its pivot value
// from the lane that holds it (a shuffle within the group) and updates the
// rows above it, and z = D^-1 t meets the row l = L_k(rho, :) in the lane's
// partial dot product.  Every entry sees the same multiply-adds in the same
// order as in the shared-memory form, so the results are the same bits.
// Qs: Q row-major, Rs: R D^-1 column-major, both leading dimension rk; y: the
// group's right-hand side (shared); lrow(b) = L_k(rho, b).
template <int NB>
__device__ __forceinline__ double group_interp(const double *Qs, const double *Rs, const double *ri,
                                               const double *y, const double *lrow, size_t lst, int rk, bool ok,
                                               double *zrow) {
  const int lane = lane_id(), gl = lane % TTQ_SG, gbase = lane & ~(TTQ_SG - 1);
  double tq[NB];
#pragma unroll
  for (int m = 0; m < NB; ++m) tq[m] = 0.0;
  for (int b = 0; b < rk; ++b) {                 // t = Q^T y
    const double yb = y[b];
    const double *Qb = Qs + b * rk + gl;
#pragma unroll
    for (int m = 0; m < NB; ++m)
      if (m < NB - 1 || gl + TTQ_SG * m < rk) tq[m] = fma(Qb[TTQ_SG * m], yb, tq[m]);
  }
#pragma unroll
  for (int m = NB - 1; m >= 0; --m) {            // back substitution: t_i -= C_ij t_j, j descending
#pragma unroll
    for (int sl = TTQ_SG - 1; sl >= 0; --sl) {
      const int jj = TTQ_SG * m + sl;
      if (jj >= rk) continue;
      const double vj = __shfl_sync(0xffffffffu, tq[m], gbase + sl);
      const double *Cj = Rs + (size_t)jj * rk + gl;
#pragma unroll
      for (int mm = 0; mm < m; ++mm) tq[mm] = fma(-Cj[TTQ_SG * mm], vj, tq[mm]);
      if (gl < sl) tq[m] = fma(-Cj[TTQ_SG * m], vj, tq[m]);
    }
  }
  double acc = 0.0;                              // L_k(rho, :) z, z = D^-1 t
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    const int b = gl + TTQ_SG * m;
    if (m < NB - 1 || b < rk) {
      const double zb = tq[m] * ri[b];
      if (ok) {
        acc = fma(lrow[(size_t)b * lst], zb, acc);
        zrow[b] = zb;
      }
    }
  }
  return acc;
}

// What one CTA needs for the random-sample stage of interface k (Alg. 2,
// first step): ranks, sizes, the counter-based stream, the factors of G_k in
// shared memory (R D^-1 column-major, Q row-major or nullptr, 1/R_jj) and the
// cross's rows and columns (excluded: the residual is zero there).
struct SampleCtx {
  int k, rk, rl, rn, Nk, Nk1, M, Ncol, S, flp;
  unsigned long long sid;
  const double *Rs, *Qs, *ri;
  const int *rset, *gset;
};

// One task of TTQ_SPW samples by one warp: each lane of the first TTQ_SPW
// draws a sample and tests the exclusion, then a group of TTQ_SG lanes per
// sample evaluates A at the point and forms E = A - L_k(rho, :) G_k^-1 y, y =
// R_{k+1}(:, gamma); every sample's z = G_k^-1 y is kept (zs), its score and
// residual stored (cs, ce).  mxw: the warp's node-index scratch, yv: the
// warp's group vectors (TTQ_SPW pairs of cap + 1).
__device__ __forceinline__ void sample_task(const Dev &D, const SampleCtx &c, int task, int (*mxw)[TTQ_SPW],
                                            double *yv, double &best, unsigned &nel, unsigned &nev,
                                            unsigned long long &fl) {
  const int lane = lane_id(), d = D.d;
  const int g = lane / TTQ_SG, gl = lane % TTQ_SG;
  const int k = c.k, rk = c.rk, rn = c.rn, Nk = c.Nk, M = c.M, Ncol = c.Ncol, S = c.S;
  const int *rset = c.rset, *gset = c.gset;
  const double *Rs = c.Rs, *Qs = c.Qs, *ri = c.ri;
  const unsigned long long sid = c.sid;
  const int flp = c.flp;
  const int vst = D.cap + 1;                         // padded group vector stride
  double *y = yv + g * 2 * vst, *t = y + vst;        // this group's y (then z) and Q^T y
  const int base = task * TTQ_SPW;
  // one lane per sample: draw and exclusion test
  int rho = 0, gam = 0, ok = 0;
  if (lane < TTQ_SPW && base + lane < S) {
    const int tt = base + lane;
    rho = draw_index(D.seed, sid, 2ULL * tt, (unsigned long long)M);
    gam = draw_index(D.seed, sid, 2ULL * tt + 1, (unsigned long long)Ncol);
    bool ex = false;
    for (int a = 0; a < rk; ++a) ex |= (rset[a] == rho) | (gset[a] == gam);
    if (ex) {
      D.cs[k][tt] = -1.0;
      D.ce[k][tt] = 0.0;
    } else {
      ok = 1;
    }
  }
  // group g takes sample base + g: its node indices, then A at the point
  rho = __shfl_sync(0xffffffffu, rho, g);
  gam = __shfl_sync(0xffffffffu, gam, g);
  ok = __shfl_sync(0xffffffffu, ok, g);
  const int alpha = rho / Nk, i = rho % Nk, j = gam / rn, beta = gam % rn;
  // every group evaluates (full-warp shuffles inside); a group without a
  // sample takes node 0 of every mode and its value is not used
  for (int v = gl; v < d; v += TTQ_SG) {
    int mv = 0;
    if (ok) {
      if (v < k - 1) mv = D.lidx[k - 1][alpha * d + v];
      else if (v == k - 1) mv = i;
      else if (v == k) mv = j;
      else mv = D.ridx[k + 1][beta * d + v];
    }
    mxw[v][g] = mv;
  }
  __syncwarp();
  double A = group_point_value<TTQ_SG>(D, &mxw[0][g], TTQ_SPW, gl);
  if (!ok) A = 0.0;
  for (int b = gl; b < rk; b += TTQ_SG) y[b] = ok ? D.Y[k + 1][core_at(D, k + 1, b, j, beta)] : 0.0;
  __syncwarp();
  const int nb = (rk + TTQ_SG - 1) / TTQ_SG;
  double acc = 0.0;                             // L_k(rho, :) G_k^-1 y
  // the sample's z = G^-1 y is kept: the best sample's is the first rook step's
  double *zrow = D.zs[k] + (size_t)(base + g) * D.cap;
  if (Qs && nb <= 8) {                          // ranks up to 8 TTQ_SG in registers
    const double *lrow = D.Y[k] + core_at(D, k, alpha, i, 0);
    const size_t lst = (size_t)D.capL[k - 1] * Nk;
    switch (nb) {
      case 8: acc = group_interp<8>(Qs, Rs, ri, y, lrow, lst, rk, ok, zrow); break;
      case 7: acc = group_interp<7>(Qs, Rs, ri, y, lrow, lst, rk, ok, zrow); break;
      case 6: acc = group_interp<6>(Qs, Rs, ri, y, lrow, lst, rk, ok, zrow); break;
      case 5: acc = group_interp<5>(Qs, Rs, ri, y, lrow, lst, rk, ok, zrow); break;
      case 4: acc = group_interp<4>(Qs, Rs, ri, y, lrow, lst, rk, ok, zrow); break;
      case 3: acc = group_interp<3>(Qs, Rs, ri, y, lrow, lst, rk, ok, zrow); break;
      case 2: acc = group_interp<2>(Qs, Rs, ri, y, lrow, lst, rk, ok, zrow); break;
      default: acc = group_interp<1>(Qs, Rs, ri, y, lrow, lst, rk, ok, zrow); break;
    }
  } else {
    for (int r0 = gl; r0 < rk; r0 += TTQ_SG) {   // t = Q^T y
      double acc = 0.0;
      if (Qs) for (int b = 0; b < rk; ++b) acc = fma(Qs[b * rk + r0], y[b], acc);
      else for (int b = 0; b < rk; ++b) acc = fma(D.Qr[k][b * D.cap + r0], y[b], acc);
      t[r0] = acc;
    }
    __syncwarp();
    for (int jj = rk - 1; jj >= 0; --jj) {        // back substitution with R D^-1: t_i -= C_ij t_j
      const double vj = t[jj];
      for (int r0 = gl; r0 < jj; r0 += TTQ_SG) t[r0] = fma(-Rs[r0 + jj * rk], vj, t[r0]);
      __syncwarp();
    }
    for (int b = gl; b < rk; b += TTQ_SG) {       // z = D^-1 t
      y[b] = t[b] * ri[b];
      if (ok) zrow[b] = y[b];
    }
    __syncwarp();
    if (ok) for (int b = gl; b < rk; b += TTQ_SG) acc = fma(D.Y[k][core_at(D, k, alpha, i, b)], y[b], acc);
  }
#pragma unroll
  for (int o = TTQ_SG / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (ok && gl == 0) {
    const int tt = base + g;
    const double E = A - acc;
    const double sc = isfinite(E) ? fabs(E) : -1.0;
    D.cs[k][tt] = sc;
    D.ce[k][tt] = E;
    ++nev;
    if (sc >= 0.0) { best = fmax(best, sc); ++nel; }
    fl += (unsigned long long)flp + 3ULL * rk * rk + 2ULL * rk + 1;
  }
  __syncwarp();
}

// Several pivots per sweep: the starts of interface k's searches, up to npiv
// samples taken one at a time as the tie-window argmax of the sample scores
// among the samples whose row and column differ from those of the starts
// already taken (the first is the sample stage_pick takes).  Whole CTA; clears
// the stage reduction; returns the count, with each start's residual.
__device__ int sample_starts(const Dev &D, int k, int *pick, double *perr) {
  __shared__ long long red[TTQ_WARPS];
  __shared__ int redi[TTQ_WARPS];
  __shared__ double rede[TTQ_WARPS];
  __shared__ int srow[TTQ_MAXP], scol[TTQ_MAXP], n_s;
  State *st = D.st;
  IfaceState &I = st->it[k];
  const int tid = threadIdx.x, nt = blockDim.x, lane = lane_id(), warp = warp_id(), nw = nt >> 5;
  const int S = D.S[k];
  const unsigned long long M = (unsigned long long)st->r[k - 1] * D.N[k - 1];
  const unsigned long long Ncol = (unsigned long long)D.N[k] * st->r[k + 1];
  const unsigned long long sid = stream_id(st->sweep, k, 1);
  const double scale = __longlong_as_double((long long)__ldcg(&st->scale_bits));
  const long long *csb = reinterpret_cast<const long long *>(D.cs[k]);
  const double *ce = D.ce[k];
  __syncthreads();
  if (tid == 0) { I.smax_bits = 0ULL; I.stage_count = 0; n_s = 0; }
  __syncthreads();
  for (int n = 0; n < D.npiv; ++n) {
    // pass 1: the largest eligible score; pass 2: the first eligible sample in the window
    long long best = -1;
    for (int t = tid; t < S; t += nt) {
      const long long v = __ldcg(csb + t);
      if (v < 0) continue;
      const int rw = (int)draw_index(D.seed, sid, 2ULL * t, M), cl = (int)draw_index(D.seed, sid, 2ULL * t + 1, Ncol);
      bool ex = false;
      for (int q = 0; q < n; ++q) ex |= (srow[q] == rw) || (scol[q] == cl);
      if (!ex && v > best) best = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      best = ob > best ? ob : best;
    }
    if (lane == 0) red[warp] = best;
    __syncthreads();
    best = red[0];
    for (int w = 1; w < nw; ++w) best = red[w] > best ? red[w] : best;
    __syncthreads();
    if (best < 0) break;                         // uniform: every thread saw the same maximum
    const double smax = __longlong_as_double(best);
    const double thr = __dadd_rn(smax, -__dadd_rn(__dmul_rn(TTQ_TIE_REL, smax), __dmul_rn(TTQ_TIE_ABS, scale)));
    const long long thrb = thr > 0.0 ? __double_as_longlong(thr) : 0LL;
    int first = 0x7fffffff;
    double ef = 0.0;
    for (int t = tid; t < S; t += nt) {
      const long long v = __ldcg(csb + t);
      if (v < thrb || t >= first) continue;
      const int rw = (int)draw_index(D.seed, sid, 2ULL * t, M), cl = (int)draw_index(D.seed, sid, 2ULL * t + 1, Ncol);
      bool ex = false;
      for (int q = 0; q < n; ++q) ex |= (srow[q] == rw) || (scol[q] == cl);
      if (!ex) { first = t; ef = __ldcg(ce + t); }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int of = __shfl_xor_sync(0xffffffffu, first, o);
      const double oe = __shfl_xor_sync(0xffffffffu, ef, o);
      if (of < first) { first = of; ef = oe; }
    }
    if (lane == 0) { redi[warp] = first; rede[warp] = ef; }
    __syncthreads();
    if (tid == 0) {
      int f = redi[0];
      double e = rede[0];
      for (int w = 1; w < nw; ++w)
        if (redi[w] < f) { f = redi[w]; e = rede[w]; }
      pick[n] = f;
      perr[n] = e;
      srow[n] = (int)draw_index(D.seed, sid, 2ULL * f, M);
      scol[n] = (int)draw_index(D.seed, sid, 2ULL * f + 1, Ncol);
      n_s = n + 1;
    }
    __syncthreads();
  }
  return n_s;
}

__global__ void __launch_bounds__(TTQ_WARPS * 32, 2) k_samples(Dev *const *Dps) {
  // descriptor read in place: its shared-memory copy would cost the kernel its
  // second resident CTA per SM (R, Q and the group vectors fill the rest)
  const Dev &D = *Dps[blockIdx.z];
  // the run flags, the ranks and the cross's parent pointers were last written
  // at the end of the previous sweep, which had completed before kernel (b)
  // passed its own wait: they are read before this kernel's wait
  State *st = D.st;
  const int k = blockIdx.y + 1;
  if (!iface_searchable(D, st, k)) return;
  __shared__ int mx[TTQ_WARPS][TTQ_MAXD][TTQ_SPW];   // node indices of the warp's points
  __shared__ int rset[TTQ_MAXR], gset[TTQ_MAXR];      // cross rows / columns (excluded)
  __shared__ double ri[TTQ_MAXR];
  __shared__ SolveSmem sc;
  extern __shared__ double fac[];
  const int lane = lane_id(), warp = warp_id();
  const int rk = st->r[k], rl = st->r[k - 1], rn = st->r[k + 1];
  const int Nk = D.N[k - 1], Nk1 = D.N[k];
  double *Rs = fac;                                  // R column-major, ld rk
  double *Qs = D.q_in_smem ? fac + (size_t)D.cap * D.cap : nullptr;   // Q row-major, ld rk
  const int vst = D.cap + 1;
  double *yv = fac + (size_t)D.cap * D.cap * (D.q_in_smem ? 2 : 1) + (size_t)warp * TTQ_SPW * 2 * vst;
  for (int a = threadIdx.x; a < rk; a += blockDim.x) {
    rset[a] = D.lpar[k][a] * Nk + D.lnode[k][a];
    gset[a] = D.rnode[k][a] * rn + D.rpar[k][a];
  }
  pdl_wait();
  pdl_release();
  // R D^-1 (column-major), Q and 1/R_jj from kernel (b), copied asynchronously
  stage_compact_async(Rs, D.Cc[k], Qs, D.Qr[k], rk, D.cap);
  for (int a = threadIdx.x; a < rk; a += blockDim.x) cp_async8(ri + a, D.rinv[k] + a);
  cp_async_wait_all();
  __syncthreads();
  const SampleCtx c = {k, rk, rl, rn, Nk, Nk1, rl * Nk, Nk1 * rn, D.S[k], point_flops(D),
                       stream_id(st->sweep, k, 1), Rs, Qs, ri, rset, gset};
  double best = 0.0;
  unsigned nel = 0, nev = 0;
  unsigned long long fl = 0;
  // tasks of TTQ_SPW samples dealt CTA-first, so the interface's CTAs (and the
  // SMs they share) carry counts that differ by one task at most
  const int ntask = (c.S + TTQ_SPW - 1) / TTQ_SPW;
  for (int task = warp * gridDim.x + blockIdx.x; task < ntask; task += gridDim.x * TTQ_WARPS)
    sample_task(D, c, task, mx[warp], yv, best, nel, nev, fl);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    nel += __shfl_xor_sync(0xffffffffu, nel, o);
    nev += __shfl_xor_sync(0xffffffffu, nev, o);
    fl += __shfl_xor_sync(0xffffffffu, fl, o);
  }
  if (lane == 0) {
    if (nev) atomicAdd(&st->it[k].evals, (unsigned long long)nev);
    if (fl) atomicAdd(&st->flops[3], fl);
    stage_publish(st->it[k], best, nel);
  }
  // the last CTA of the interface takes the best sample and the first column solve
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    sc.is_last = (atomicAdd(&st->it[k].items_done, 1u) == gridDim.x - 1) ? 1 : 0;
    if (sc.is_last) st->it[k].items_done = 0;
  }
  __syncthreads();
  if (!sc.is_last) return;
  __threadfence();
  if (D.npiv == 1) {
    stage_finish(D, k, 0, 0, Rs, Qs, ri, sc);
  } else {
    __shared__ int picks[TTQ_MAXP];
    __shared__ double perrs[TTQ_MAXP];
    const int n = sample_starts(D, k, picks, perrs);
    for (int j = 0; j < n; ++j) stage_finish(D, k, j, 0, Rs, Qs, ri, sc, false, picks[j], perrs[j]);
  }
}

// Work list of a rook step over every interface of the instance: lane k-1
// holds interface k's item count; prefix sums over the lanes.
struct ItemMap {
  int pre, cnt, total;
};
__device__ __forceinline__ ItemMap item_map(int cnt) {
  const int lane = lane_id();
  int pre = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, pre, o);
    if (lane >= o) pre += v;
  }
  return {pre, cnt, __shfl_sync(0xffffffffu, pre, 31)};
}

// Rook kernels: resident CTAs per SM (registers for the loads in flight) and the
// unroll of the product over the rank, which sets how many L_k rows a warp has
// requested ahead of its multiply-adds
#ifndef TTQ_ROOK_CTAS
#define TTQ_ROOK_CTAS 2
#endif
#ifndef TTQ_ROOK_UNROLL
#define TTQ_ROOK_UNROLL 8
#endif
constexpr int kRookUnroll = TTQ_ROOK_UNROLL;
constexpr int kRookUnroll2 = TTQ_ROOK_UNROLL / 2;   // the same depth in pairs of rank steps

// Score of a residual for the argmax, as IEEE bits: |E| for finite E (non-negative
// doubles order like their bit patterns), else none.  Integer operations only.
__device__ __forceinline__ bool score_bits(double E, unsigned long long &bits) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(E) & 0x7fffffffffffffffULL;
  bits = b;
  return b < 0x7ff0000000000000ULL;             // finite
}

// One work item of the column step: rows rho = (alpha, i), i in [i0, i1) with
// NQ rows of 32 nodes per lane.  E = A(rho, gamma*) - L_k(rho, :) z.
template <int NQ>
__device__ __forceinline__ void col_item(const Dev &D, int k, int j, int alpha, int i0, int i1, int rk, const int *ms,
                                         const FiberU &u, const double *pl, const int *exc, int nex, const double *z,
                                         unsigned long long (&bq)[NQ], unsigned &nel, unsigned &nev) {
  const double *tab = uses_ptab(D, rk) ? ptab_of(D, k, j) : nullptr;
  double *csj = cs_of(D, k, j), *cej = ce_of(D, k, j);
  const int lane = lane_id(), Nk = D.N[k - 1];
  int iq[NQ];
  bool ok[NQ];
  double A[NQ], acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    iq[q] = i0 + lane + 32 * q;
    bool ex = false;
    for (int e = 0; e < nex; ++e) ex |= (exc[e] == iq[q]);
    ok[q] = iq[q] < i1 && !ex;
    A[q] = !ok[q] ? 0.0
           : (tab ? fiber_value_tab(D, k - 1, ms, u, iq[q], tab, 0, k - 1) : fiber_value(D, k - 1, ms, u, pl, iq[q]));
    acc[q] = 0.0;
  }
  {
    const double *Yc = D.Y[k] + core_at(D, k, alpha, 0, 0);
    const size_t cst = (size_t)D.capL[k - 1] * Nk;
    int c[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) c[q] = min(iq[q], Nk - 1);
    // z two entries per shared-memory load; the products still added in rank order
    int b = 0;
#pragma unroll kRookUnroll2
    for (; b + 1 < rk; b += 2) {
      const double2 zz = *reinterpret_cast<const double2 *>(z + b);
      const double *row = Yc + b * cst;
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[q] = fma(row[c[q]], zz.x, acc[q]);
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[q] = fma(row[cst + c[q]], zz.y, acc[q]);
    }
    if (b < rk) {
      const double zb = z[b];
      const double *row = Yc + b * cst;
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[q] = fma(row[c[q]], zb, acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    bq[q] = 0ULL;                                  // score bits + 1 of the row's eligible candidate, 0: none
    if (iq[q] >= i1) continue;
    const int rho = alpha * Nk + iq[q];
    if (!ok[q]) { csj[rho] = -1.0; cej[rho] = 0.0; continue; }
    const double E = A[q] - acc[q];
    unsigned long long sb;
    const bool fin = score_bits(E, sb);
    csj[rho] = fin ? __longlong_as_double((long long)sb) : -1.0;
    cej[rho] = E;
    ++nev;
    if (fin) { bq[q] = sb + 1ULL; ++nel; }
  }
}

// One work item of the row step: columns gamma = (j, beta), j in [j0, j1).
// E = A(rho*, gamma) - l^T R_{k+1}(:, gamma) with z = G^-T l.
template <int NQ>
__device__ __forceinline__ void row_item(const Dev &D, int k, int j, int beta, int j0, int j1, int rk, int rn,
                                         const int *ms, const FiberU &u, const double *pl, const int *exc, int nex,
                                         const double *z, unsigned long long (&bq)[NQ], unsigned &nel, unsigned &nev) {
  const double *tab = uses_ptab(D, rk) ? ptab_of(D, k, j) : nullptr;
  double *csj = cs_of(D, k, j), *cej = ce_of(D, k, j);
  const int lane = lane_id(), Nk1 = D.N[k];
  int jq[NQ];
  bool ok[NQ];
  double A[NQ], acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    jq[q] = j0 + lane + 32 * q;
    bool ex = false;
    for (int e = 0; e < nex; ++e) ex |= (exc[e] == jq[q]);
    ok[q] = jq[q] < j1 && !ex;
    A[q] = !ok[q] ? 0.0 : (tab ? fiber_value_tab(D, k, ms, u, jq[q], tab, k + 1, D.d) : fiber_value(D, k, ms, u, pl, jq[q]));
    acc[q] = 0.0;
  }
  {
    const double *Yr = D.Y[k + 1] + core_at(D, k + 1, 0, 0, beta);
    int c[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) c[q] = min(jq[q], Nk1 - 1);
    int a = 0;
#pragma unroll kRookUnroll2
    for (; a + 1 < rk; a += 2) {
      const double2 zz = *reinterpret_cast<const double2 *>(z + a);
      const double *row = Yr + (size_t)a * Nk1;
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[q] = fma(row[c[q]], zz.x, acc[q]);
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[q] = fma(row[Nk1 + c[q]], zz.y, acc[q]);
    }
    if (a < rk) {
      const double za = z[a];
      const double *row = Yr + (size_t)a * Nk1;
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[q] = fma(row[c[q]], za, acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    bq[q] = 0ULL;
    if (jq[q] >= j1) continue;
    const int g = jq[q] * rn + beta;
    if (!ok[q]) { csj[g] = -1.0; cej[g] = 0.0; continue; }
    const double E = A[q] - acc[q];
    unsigned long long sb;
    const bool fin = score_bits(E, sb);
    csj[g] = fin ? __longlong_as_double((long long)sb) : -1.0;
    cej[g] = E;
    ++nev;
    if (fin) { bq[q] = sb + 1ULL; ++nel; }
  }
}

// warp totals of a stretch of NQ rows: evaluations, each row's maximum (stored
// at its slot outer * rows + row, the order of the candidate indices, -1 when
// the row has no eligible candidate) and the stage reduction (pass 1 of the argmax)
template <int NQ>
__device__ __forceinline__ void rows_publish(const Dev &D, IfaceState &I, int k, int j, int slot0,
                                             unsigned long long (&bq)[NQ], unsigned nel, unsigned nev) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bq[q], o);
      bq[q] = ob > bq[q] ? ob : bq[q];
    }
    nel += __shfl_xor_sync(0xffffffffu, nel, o);
    nev += __shfl_xor_sync(0xffffffffu, nev, o);
  }
  if (lane_id() == 0) {
    unsigned long long best = 0ULL;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      im_of(D, k, j)[slot0 + q] = bq[q] ? __longlong_as_double((long long)(bq[q] - 1ULL)) : -1.0;
      best = bq[q] > best ? bq[q] : best;
    }
    if (nev) atomicAdd(&I.evals, (unsigned long long)nev);
    if (nel) {
      atomicMax(&I.smax_bits, best - 1ULL);
      atomicAdd(&I.stage_count, nel);
    }
  }
}

// Work of a rook step.  Its unit is a row: 32 candidates of one fiber (one
// outer index) of one searching interface, in the order of the candidate
// indices.  Two deals, decided alike by every CTA:
//  - items: fibers split into chunks of R rows (R in 1, 2, 4, the smallest whose
//    items fit in one wave of the grid's warps), one item per warp at most,
//    walked chunk-major; when the items fit, every warp meets one chain of
//    dependent loads and setup (the latency of low-rank steps);
//  - stretches, when even 4-row items overflow one wave: every warp takes a
//    contiguous stretch of rows of near-equal length (they differ by one row at
//    most), processed in pieces of at most four rows that stop at fiber ends,
//    so every scheduler of every SM gets the same share of the FP64 work and
//    no sparse second wave of items trails the first.
// Lane k-1 of the warp holds interface k's outer rank and nodes; pieces come
// out as (interface, outer index, first row, rows).
// the searches of interface k that run the rook step (bit j: search j).  With
// several searches, one that meets an earlier running search at this step
// (stage 1, a column step: the same column to search; stage 2, a row step:
// the same row) stops: from here both take the same steps and end on the same
// pivot, which the acceptance would drop as a repeat.  Those go to *newly.
template <bool MULTI>
__device__ __forceinline__ unsigned running_searches(const Dev &D, State *st, int k, int stage,
                                                     unsigned *newly = nullptr) {
  unsigned m = 0, mg = 0;
  int pos[TTQ_MAXP] = {-1, -1, -1, -1};
  for (int j = 0; j < (MULTI ? D.npiv : 1); ++j) {
    const IfaceState &I = search_state(D, st, k, j);
    if (!I.active || I.rook_done) continue;
    if constexpr (MULTI) {
      if (I.merged) continue;
      const int p = stage == 1 ? I.col : I.row;
      bool meet = false;
      for (int q = 0; q < j; ++q) meet |= ((m >> q) & 1u) && pos[q] == p;
      pos[j] = p;
      if (meet) {
        mg |= 1u << j;
        continue;
      }
    }
    m |= 1u << j;
  }
  if (newly) *newly = mg;
  return m;
}
// the searches of interface k that met an earlier one (bits of m) stop: the
// decisions kernel after this step and the acceptance skip them
__device__ __forceinline__ void mark_met(const Dev &D, State *st, int k, unsigned m) {
  for (int j = 0; j < TTQ_MAXP; ++j)
    if ((m >> j) & 1u) search_state(D, st, k, j).merged = 1;
}
// the n-th (from 0) set bit of m
__device__ __forceinline__ int nth_search(unsigned m, int n) {
  for (int j = 0; j < TTQ_MAXP; ++j)
    if ((m >> j) & 1u) {
      if (n == 0) return j;
      --n;
    }
  return 0;
}

struct RookDeal {
  ItemMap im;
  int R, pos, end;
  bool items;
};
__device__ __forceinline__ RookDeal rook_deal(const Dev &D, int outer, int Nl, int rmax) {
  const long long W = (long long)gridDim.x * TTQ_WARPS;
  RookDeal q;
  q.R = rows_per_item(outer, Nl, rmax);
  q.im = item_map(outer ? outer * node_chunks(Nl, q.R).nch : 0);
  q.items = q.im.total <= W;
  if (!q.items) q.im = item_map(outer ? outer * ((Nl + 31) >> 5) : 0);
  const long long g = (long long)deal_slot(warp_id(), D.sms, q.im.total) * gridDim.x + blockIdx.x;
  if (q.items) {
    q.pos = (int)g;
    q.end = g < q.im.total ? (int)g + 1 : (int)g;
  } else {
    q.pos = (int)(g * q.im.total / W);
    q.end = (int)((g + 1) * q.im.total / W);
  }
  return q;
}
// the next piece: interface k, outer index o (of outer rank ok), rows [q0, q0 + nq) of N nodes
__device__ __forceinline__ void rook_piece(RookDeal &q, int k, int ok, int N, int &o, int &q0, int &nq) {
  const int local = q.pos - __shfl_sync(0xffffffffu, q.im.pre - q.im.cnt, k - 1);
  if (q.items) {
    const NodeChunks nc = node_chunks(N, q.R);
    const int ch = local / ok;
    o = local % ok;
    q0 = ch * nc.base + min(ch, nc.extra);
    nq = nc.base + (ch < nc.extra ? 1 : 0);
    q.pos += 1;
  } else {
    const int rows = (N + 31) >> 5;
    o = local / rows;
    q0 = local % rows;
    nq = min(min(4, rows - q0), q.end - q.pos);
    q.pos += nq;
  }
}

// One piece of the column step of interface k (one warp): rows rho = (alpha,
// i) for the nq rows of 32 nodes from q0 of fiber alpha, E = A(rho, gamma*) -
// L_k(rho, :) z, z = G_k^-1 R_{k+1}(:, gamma*) (zvec, copied to the warp's
// shared vector when zk != k), candidates and per-row maxima stored, pass 1 of
// the argmax.  The piece's loads form one round: z, the fiber's left indices,
// the fixed right indices (I.fix), the cross's parent pointers.
__device__ __forceinline__ void col_piece(const Dev &D, State *st, RookSmem &sh, int k, int j, int alpha, int q0,
                                          int nq, int rk, int &zk, unsigned long long &fl) {
  const int lane = lane_id(), warp = warp_id(), d = D.d;
  IfaceState &I = search_state(D, st, k, j);
  const int zkey = k + 64 * j;
  const int Nk = D.N[k - 1], rows = (Nk + 31) >> 5;
  const int i0 = 32 * q0, i1 = min(Nk, 32 * (q0 + nq)), slot0 = alpha * rows + q0;
  double zr[TTQ_MAXR / 32];
  int lp[TTQ_MAXR / 32], ln[TTQ_MAXR / 32];
  const bool newz = zkey != zk;
  const double *zsrc = zvec_of(D, k, j);
#pragma unroll
  for (int q = 0; q < TTQ_MAXR / 32; ++q) {
    const int a = lane + 32 * q;
    zr[q] = (newz && a < rk) ? __ldcg(zsrc + a) : 0.0;
    lp[q] = a < rk ? D.lpar[k][a] : -1;
    ln[q] = a < rk ? D.lnode[k][a] : 0;
  }
  const int vl = (lane < k - 1) ? D.lidx[k - 1][alpha * d + lane] : 0;
  const int vr = (lane >= k && lane < d) ? __ldcg(I.fix + lane) : 0;
  if (newz) {
#pragma unroll
    for (int q = 0; q < TTQ_MAXR / 32; ++q)
      if (lane + 32 * q < rk) sh.z[warp][lane + 32 * q] = zr[q];
    zk = zkey;
  }
  if (lane < d) sh.ms[warp][lane] = (lane < k - 1) ? vl : vr;
  // rows of the cross with this parent alpha: excluded nodes i
  int nex = 0;
#pragma unroll
  for (int q = 0; q < TTQ_MAXR / 32; ++q) {
    const bool hit = lp[q] == alpha;
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    if (hit) sh.exc[warp][nex + __popc(bal & ((1u << lane) - 1))] = ln[q];
    nex += __popc(bal);
  }
  __syncwarp();
  FiberU u = fiber_setup(D, k - 1, sh.ms[warp], sh.pl[warp]);
  // per node: the entry (the shared right-mode factors come from the step's table), the product, the residual
  const int tabbed = uses_ptab(D, rk) ? (d - k) - 1 : 0;
  fl += (unsigned long long)u.fl_uniform + (unsigned long long)(i1 - i0) * (u.fl_node - tabbed + 2 * rk + 1);
  unsigned nel = 0, nev = 0;
#define TTQ_COL_PIECE(Q)                                                                                      \
  {                                                                                                           \
    unsigned long long bq[Q];                                                                                 \
    col_item<Q>(D, k, j, alpha, i0, i1, rk, sh.ms[warp], u, sh.pl[warp], sh.exc[warp], nex, sh.z[warp], bq,   \
                nel, nev);                                                                                    \
    rows_publish<Q>(D, I, k, j, slot0, bq, nel, nev);                                                         \
  }
  switch (nq) {
    case 4: TTQ_COL_PIECE(4) break;
    case 3: TTQ_COL_PIECE(3) break;
    case 2: TTQ_COL_PIECE(2) break;
    default: TTQ_COL_PIECE(1) break;
  }
#undef TTQ_COL_PIECE
  __syncwarp();
}

// Alg. 2, column step: E(:, gamma*) over all rows rho = (alpha, i) of every
// searching interface; pass 1 of the argmax per interface (pass 2 in k_solve).
// rmax: the largest item (rows of 32 candidates) of the item deal (1, 2 or 4)
template <bool MULTI>
__global__ void __launch_bounds__(TTQ_WARPS * 32, TTQ_ROOK_CTAS) k_rook_col(Dev *const *Dps, int rmax) {
  __shared__ Dev sD;
  const Dev &D = stage_dev(Dps, sD);
  pdl_wait();
  pdl_release();
  State *st = D.st;
  __shared__ RookSmem sh;
  const int lane = lane_id(), d = D.d;
  // one round of loads: the run's flags and, lane k-1, interface k's search
  // state and the ranks around it
  const int stop = st->stop, search = st->search;
  unsigned act = 0;
  int r0 = 0, r1 = 0, Nl = 1;
  unsigned met = 0;
  if (lane < d - 1) {
    act = running_searches<MULTI>(D, st, lane + 1, 1, &met);
    r0 = st->r[lane];
    r1 = st->r[lane + 1];
    Nl = D.N[lane];
  }
  if (stop || !search) return;
  if (MULTI && met && blockIdx.x == 0 && warp_id() == 0) mark_met(D, st, lane + 1, met);
  // an interface's running searches take consecutive blocks of its outer indices
  const int outer = __popc(act) * r0;
  RookDeal dl = rook_deal(D, outer, Nl, rmax);
  unsigned long long fl = 0;
  int zk = 0;                                   // interface and search whose z sits in sh.z[warp]
  while (dl.pos < dl.end) {
    const unsigned ball = __ballot_sync(0xffffffffu, lane < d - 1 && dl.im.pre > dl.pos);
    const int k = __ffs(ball);                  // interface (1-based)
    const int rk = __shfl_sync(0xffffffffu, r1, k - 1), rl = __shfl_sync(0xffffffffu, r0, k - 1);
    const unsigned am = __shfl_sync(0xffffffffu, act, k - 1);
    int o, q0, nq;
    rook_piece(dl, k, MULTI ? __popc(am) * rl : rl, D.N[k - 1], o, q0, nq);
    if constexpr (MULTI) col_piece(D, st, sh, k, nth_search(am, o / rl), o % rl, q0, nq, rk, zk, fl);
    else col_piece(D, st, sh, k, 0, o, q0, nq, rk, zk, fl);
  }
  if (lane == 0 && fl) atomicAdd(&st->flops[4], fl);
}

// One piece of the row step of interface k (one warp): columns gamma = (j,
// beta) for the nq rows of 32 nodes j from q0 of fiber beta, E = A(rho*, gamma)
// - l^T R_{k+1}(:, gamma) with z = G_k^-T l; as col_piece.
__device__ __forceinline__ void row_piece(const Dev &D, State *st, RookSmem &sh, int k, int j, int beta, int q0,
                                          int nq, int rk, int rn, int &zk, unsigned long long &fl) {
  const int lane = lane_id(), warp = warp_id(), d = D.d;
  IfaceState &I = search_state(D, st, k, j);
  const int zkey = k + 64 * j;
  const int Nk1 = D.N[k], rows = (Nk1 + 31) >> 5;
  const int j0 = 32 * q0, j1 = min(Nk1, 32 * (q0 + nq)), slot0 = beta * rows + q0;
  double zr[TTQ_MAXR / 32];
  int rp[TTQ_MAXR / 32], rnd[TTQ_MAXR / 32];
  const bool newz = zkey != zk;
  const double *zsrc = zvec_of(D, k, j);
#pragma unroll
  for (int q = 0; q < TTQ_MAXR / 32; ++q) {
    const int b = lane + 32 * q;
    zr[q] = (newz && b < rk) ? __ldcg(zsrc + b) : 0.0;
    rp[q] = b < rk ? D.rpar[k][b] : -1;
    rnd[q] = b < rk ? D.rnode[k][b] : 0;
  }
  const int vr = (lane > k && lane < d) ? D.ridx[k + 1][beta * d + lane] : 0;
  const int vl = (lane < k) ? __ldcg(I.fix + lane) : 0;
  if (newz) {
#pragma unroll
    for (int q = 0; q < TTQ_MAXR / 32; ++q)
      if (lane + 32 * q < rk) sh.z[warp][lane + 32 * q] = zr[q];
    zk = zkey;
  }
  if (lane < d) sh.ms[warp][lane] = (lane < k) ? vl : vr;
  int nex = 0;
#pragma unroll
  for (int q = 0; q < TTQ_MAXR / 32; ++q) {
    const bool hit = rp[q] == beta;
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    if (hit) sh.exc[warp][nex + __popc(bal & ((1u << lane) - 1))] = rnd[q];
    nex += __popc(bal);
  }
  __syncwarp();
  FiberU u = fiber_setup(D, k, sh.ms[warp], sh.pl[warp]);
  const int tabbed = uses_ptab(D, rk) ? k - 1 : 0;
  fl += (unsigned long long)u.fl_uniform + (unsigned long long)(j1 - j0) * (u.fl_node - tabbed + 2 * rk + 1);
  unsigned nel = 0, nev = 0;
#define TTQ_ROW_PIECE(Q)                                                                                           \
  {                                                                                                                \
    unsigned long long bq[Q];                                                                                      \
    row_item<Q>(D, k, j, beta, j0, j1, rk, rn, sh.ms[warp], u, sh.pl[warp], sh.exc[warp], nex, sh.z[warp], bq,     \
                nel, nev);                                                                                         \
    rows_publish<Q>(D, I, k, j, slot0, bq, nel, nev);                                                              \
  }
  switch (nq) {
    case 4: TTQ_ROW_PIECE(4) break;
    case 3: TTQ_ROW_PIECE(3) break;
    case 2: TTQ_ROW_PIECE(2) break;
    default: TTQ_ROW_PIECE(1) break;
  }
#undef TTQ_ROW_PIECE
  __syncwarp();
}

// Alg. 2, row step: E(rho*, :) over all columns gamma = (j, beta) of every
// searching interface, rows of 32 nodes j of the fibers beta, dealt like the
// column step's; pass 1 of the argmax.
template <bool MULTI>
__global__ void __launch_bounds__(TTQ_WARPS * 32, TTQ_ROOK_CTAS) k_rook_row(Dev *const *Dps, int rmax) {
  __shared__ Dev sD;
  const Dev &D = stage_dev(Dps, sD);
  pdl_wait();
  pdl_release();
  State *st = D.st;
  __shared__ RookSmem sh;
  const int lane = lane_id(), d = D.d;
  const int stop = st->stop, search = st->search;
  unsigned act = 0;
  int r1 = 0, r2 = 0, Nl = 1;
  unsigned met = 0;
  if (lane < d - 1) {
    act = running_searches<MULTI>(D, st, lane + 1, 2, &met);
    r1 = st->r[lane + 1];
    r2 = st->r[lane + 2];
    Nl = D.N[lane + 1];
  }
  if (stop || !search) return;
  if (MULTI && met && blockIdx.x == 0 && warp_id() == 0) mark_met(D, st, lane + 1, met);
  const int outer = __popc(act) * r2;
  RookDeal dl = rook_deal(D, outer, Nl, rmax);
  unsigned long long fl = 0;
  int zk = 0;
  while (dl.pos < dl.end) {
    const unsigned ball = __ballot_sync(0xffffffffu, lane < d - 1 && dl.im.pre > dl.pos);
    const int k = __ffs(ball);
    const int rk = __shfl_sync(0xffffffffu, r1, k - 1), rn = __shfl_sync(0xffffffffu, r2, k - 1);
    const unsigned am = __shfl_sync(0xffffffffu, act, k - 1);
    int o, q0, nq;
    rook_piece(dl, k, MULTI ? __popc(am) * rn : rn, D.N[k], o, q0, nq);
    if constexpr (MULTI) row_piece(D, st, sh, k, nth_search(am, o / rn), o % rn, q0, nq, rk, rn, zk, fl);
    else row_piece(D, st, sh, k, 0, o, q0, nq, rk, rn, zk, fl);
  }
  if (lane == 0 && fl) atomicAdd(&st->flops[5], fl);
}

// ---------------------------------------------------------------------------
// Persistent search (one instance): the whole of Alg. 2 on every interface of
// a sweep in one cooperative launch, without kernel boundaries between its
// stages.  Every CTA belongs to the group of one interface for the whole
// launch (groups sized by the interface's expected work: samples S_k (3 r_k^2)
// plus the rook rows (r_{k-1} N_k + N_{k+1} r_{k+1}) (2 r_k)), and each group
// runs its interface's stages by itself: random samples, then up to rook_max
// column / row rounds.  A stage's CTAs deal its rows (or sample tasks) among
// themselves; each CTA arrives on the interface's counter when its share is
// done, and the last to arrive takes the stage's decisions (stage_finish:
// argmax pass 2, the rook test, the next solve, with the factors of G_k that
// every CTA of the group holds in shared memory) and publishes them by
// raising the interface's epoch; the group's other CTAs wait for that epoch.
// The CTA whose decisions end the interface's search appends its pivot.  The
// ranks, stopping rules and the sweep count follow in k_sweep_end.
//
// Every wait is bounded: past D.wait_ns of %globaltimer after the launch
// began, the waiting CTA sets st->search_abort and leaves, and every other
// wait sees the flag and leaves too; the sweep then ends with status TIMEOUT.
// The grid is the device's resident CTA slots less the two the contraction
// takes on the second stream, so in a correct run every CTA is resident and no
// wait depends on a CTA that is not running; were one held back (another
// kernel on the device), its group would wait until it runs, at most the limit.

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Interface state written by another CTA of the launch is read through L2
// (__ldcg): the L1 of this SM may hold a copy older than the writer's stores.
__device__ __forceinline__ bool iface_running(const IfaceState &I) {
  return __ldcg(&I.active) && !__ldcg(&I.rook_done);
}

// whole CTA: wait until interface k's epoch reaches e; false if the search was
// abandoned (by this wait's limit or another CTA's)
__device__ bool group_wait(State *st, int k, unsigned e, unsigned long long deadline) {
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    volatile unsigned *ep = &st->it[k].epoch;
    volatile int *ab = &st->search_abort;
    int ok = 1;
    while (*ep < e) {
      if (*ab) { ok = 0; break; }
      if (global_ns() > deadline) { atomicExch(&st->search_abort, 1); ok = 0; break; }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// whole CTA: this CTA's share of the stage is done; true in the last of the
// group's g CTAs to arrive (which then sees every other CTA's writes)
__device__ bool group_arrive(State *st, int k, int g) {
  __shared__ int last_s;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned old = atomicAdd(&st->it[k].items_done, 1u);
    last_s = (old == (unsigned)g - 1) ? 1 : 0;
    if (last_s) st->it[k].items_done = 0;
  }
  __syncthreads();
  if (last_s) __threadfence();
  return last_s != 0;
}

// whole CTA (the finisher): publish the stage's decisions
__device__ void group_publish(State *st, int k, unsigned e) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicExch(&st->it[k].epoch, e);
}

// Interface k's share of the launch's CTAs (k = 1..d-1; 0 for an interface
// that does not search) and its first CTA; the same in every CTA.
__device__ void search_groups(const Dev &D, const State *st, int G, int *first, int *count) {
  const int d = D.d, ni = d - 1;
  double w[TTQ_MAXD];
  double W = 0.0;
  int na = 0;
  for (int k = 1; k <= ni; ++k) {
    w[k] = 0.0;
    if (!iface_searchable(D, st, k)) continue;
    const double rk = st->r[k];
    const double rows = (double)st->r[k - 1] * D.N[k - 1] + (double)D.N[k] * st->r[k + 1];
    w[k] = (double)D.S[k] * (3.0 * rk * rk + 64.0) + (double)D.rook_max * rows * (2.0 * rk + 32.0);
    W += w[k];
    ++na;
  }
  int used = 0;
  for (int k = 1; k <= ni; ++k) {
    count[k] = (w[k] > 0.0) ? 1 + (int)floor((double)(G - na) * w[k] / W) : 0;
    used += count[k];
  }
  // CTAs left by the rounding go one each to the heaviest interfaces (ties: lowest k)
  while (used < G && na > 0) {
    int best = 0;
    for (int k = 1; k <= ni; ++k)
      if (w[k] > 0.0 && (best == 0 || w[k] > w[best])) best = k;
    for (int k = 1; k <= ni && used < G; ++k)
      if (w[k] > 0.0 && w[k] >= w[best]) { count[k]++; used++; }
    if (used < G)
      for (int k = 1; k <= ni && used < G; ++k)
        if (w[k] > 0.0) { count[k]++; used++; }
  }
  int o = 0;
  for (int k = 1; k <= ni; ++k) { first[k] = o; o += count[k]; }
}

// Deal of one interface's rook-step rows over its group's W = g * TTQ_WARPS
// warps (warp slot w = warp * g + gi, CTA-first): items of R rows (R = 1, 2,
// 4, the smallest whose items fit one wave of the group's warps), else
// balanced contiguous stretches in pieces of at most four rows that stop at
// fiber ends.  Pieces come out as (outer index, first row, rows).
struct GroupDeal {
  int R, pos, end;
  bool items;
};
__device__ __forceinline__ GroupDeal group_deal(int outer, int N, int g, int gi) {
  const long long W = (long long)g * TTQ_WARPS;
  GroupDeal q;
  int R = 1;
  for (; R < 4; R *= 2)
    if ((long long)outer * node_chunks(N, R).nch <= W) break;
  q.R = R;
  const long long items = (long long)outer * node_chunks(N, R).nch;
  q.items = items <= W;
  const long long total = q.items ? items : (long long)outer * ((N + 31) >> 5);
  const long long w = (long long)warp_id() * g + gi;
  if (q.items) {
    q.pos = (int)w;
    q.end = w < total ? (int)w + 1 : (int)w;
  } else {
    q.pos = (int)(w * total / W);
    q.end = (int)((w + 1) * total / W);
  }
  return q;
}
__device__ __forceinline__ void group_piece(GroupDeal &q, int outer, int N, int &o, int &q0, int &nq) {
  const int local = q.pos;
  if (q.items) {
    const NodeChunks nc = node_chunks(N, q.R);
    const int ch = local / outer;
    o = local % outer;
    q0 = ch * nc.base + min(ch, nc.extra);
    nq = nc.base + (ch < nc.extra ? 1 : 0);
    q.pos += 1;
  } else {
    const int rows = (N + 31) >> 5;
    o = local / rows;
    q0 = local % rows;
    nq = min(min(4, rows - q0), q.end - q.pos);
    q.pos += nq;
  }
}

__global__ void __launch_bounds__(TTQ_WARPS * 32, TTQ_ROOK_CTAS) k_search(Dev *const *Dps) {
  // descriptor read in place (as in k_samples): shared memory holds the
  // factors of G_k and the stage scratch, two CTAs per SM at rank cap 64
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  const unsigned long long deadline = global_ns() + D.wait_ns;
  if (st->stop || !st->search) return;
  __shared__ int first_s[TTQ_MAXD], count_s[TTQ_MAXD];
  __shared__ int mx[TTQ_WARPS][TTQ_MAXD][TTQ_SPW];
  __shared__ int rset[TTQ_MAXR], gset[TTQ_MAXR];
  __shared__ double ri[TTQ_MAXR];
  __shared__ SolveSmem sc;
  extern __shared__ double fac[];
  if (threadIdx.x == 0) search_groups(D, st, gridDim.x, first_s, count_s);
  __syncthreads();
  int k = 0;
  for (int q = 1; q <= D.d - 1; ++q)
    if (count_s[q] > 0 && (int)blockIdx.x >= first_s[q] && (int)blockIdx.x < first_s[q] + count_s[q]) k = q;
  // the ranks and run flags were written by the previous sweep's end; the
  // interface states (reset) and the factors come from kernel (b): waited for
  pdl_wait();
  if (k == 0) return;                            // CTAs beyond every group (none when all are dealt)
  const int g = count_s[k], gi = blockIdx.x - first_s[k];
  const int lane = lane_id(), warp = warp_id();
  IfaceState &I = st->it[k];
  const int rk = st->r[k], rl = st->r[k - 1], rn = st->r[k + 1];
  const int Nk = D.N[k - 1], Nk1 = D.N[k];
  // the row solves read D^-1 R and Q column-major from global memory: the
  // group pulls them into L2 now, a row per CTA in turn
  for (int a = gi; a < rk; a += g)
    for (int c = 16 * threadIdx.x; c < rk; c += 16 * blockDim.x) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(D.Sr[k] + (size_t)a * D.cap + c));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(D.Qc[k] + (size_t)a * D.cap + c));
    }
  const size_t cc = (size_t)D.cap * D.cap;
  double *Rs = fac;                              // R D^-1 column-major, ld rk (whole launch)
  double *Qs = D.q_in_smem ? fac + cc : nullptr; // Q row-major, ld rk (whole launch)
  double *scratch = fac + cc * (D.q_in_smem ? 2 : 1);   // samples' group vectors, then the rook scratch
  RookSmem &sh = *reinterpret_cast<RookSmem *>(scratch);
  stage_compact_async(Rs, D.Cc[k], Qs, D.Qr[k], rk, D.cap);
  for (int a = threadIdx.x; a < rk; a += blockDim.x) {
    cp_async8(ri + a, D.rinv[k] + a);
    rset[a] = D.lpar[k][a] * Nk + D.lnode[k][a];
    gset[a] = D.rnode[k][a] * rn + D.rpar[k][a];
  }
  cp_async_wait_all();
  __syncthreads();

  // stage 0: random samples (Alg. 2, first step), tasks dealt CTA-first in the group
  {
    const SampleCtx c = {k, rk, rl, rn, Nk, Nk1, rl * Nk, Nk1 * rn, D.S[k], point_flops(D),
                         stream_id(st->sweep, k, 1), Rs, Qs, ri, rset, gset};
    double *yv = scratch + (size_t)warp * TTQ_SPW * 2 * (D.cap + 1);
    double best = 0.0;
    unsigned nel = 0, nev = 0;
    unsigned long long fl = 0;
    const int ntask = (c.S + TTQ_SPW - 1) / TTQ_SPW;
    for (int task = warp * g + gi; task < ntask; task += g * TTQ_WARPS)
      sample_task(D, c, task, mx[warp], yv, best, nel, nev, fl);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
      nel += __shfl_xor_sync(0xffffffffu, nel, o);
      nev += __shfl_xor_sync(0xffffffffu, nev, o);
      fl += __shfl_xor_sync(0xffffffffu, fl, o);
    }
    if (lane == 0) {
      if (nev) atomicAdd(&I.evals, (unsigned long long)nev);
      if (fl) atomicAdd(&st->flops[3], fl);
      stage_publish(I, best, nel);
    }
  }
  if (group_arrive(st, k, g)) {
    stage_finish(D, k, 0, 0, Rs, Qs, ri, sc);
    if (!iface_running(I)) sweep_append(D, st, k);
    group_publish(st, k, 1u);
  }
  unsigned e = 1;
  unsigned long long fl_col = 0, fl_row = 0;
  for (int round = 0; round < D.rook_max; ++round) {
    // column step: E(:, gamma*) over the rows rho = (alpha, i), alpha < r_{k-1}
    if (!group_wait(st, k, e, deadline)) break;
    if (!iface_running(I)) break;
    {
      int zk = 0;
      GroupDeal q = group_deal(rl, Nk, g, gi);
      while (q.pos < q.end) {
        int alpha, q0, nq;
        group_piece(q, rl, Nk, alpha, q0, nq);
        col_piece(D, st, sh, k, 0, alpha, q0, nq, rk, zk, fl_col);
      }
    }
    ++e;
    if (group_arrive(st, k, g)) {
      stage_finish(D, k, 0, 1, nullptr, nullptr, ri, sc);
      if (!iface_running(I)) sweep_append(D, st, k);
      group_publish(st, k, e);
    }
    // row step: E(rho*, :) over the columns gamma = (j, beta), beta < r_{k+1}
    if (!group_wait(st, k, e, deadline)) break;
    if (!iface_running(I)) break;
    {
      int zk = 0;
      GroupDeal q = group_deal(rn, Nk1, g, gi);
      while (q.pos < q.end) {
        int beta, q0, nq;
        group_piece(q, rn, Nk1, beta, q0, nq);
        row_piece(D, st, sh, k, 0, beta, q0, nq, rk, rn, zk, fl_row);
      }
    }
    ++e;
    if (group_arrive(st, k, g)) {
      stage_finish(D, k, 0, 2, Rs, Qs, ri, sc);
      if (!iface_running(I)) sweep_append(D, st, k);
      group_publish(st, k, e);
    }
  }
  if (lane == 0) {
    if (fl_col) atomicAdd(&st->flops[4], fl_col);
    if (fl_row) atomicAdd(&st->flops[5], fl_row);
  }
}

// The end of a sweep whose search ran in k_search (one CTA, after the
// contraction has joined): ranks, evaluations, stopping rules, sweep count and
// the WHILE condition (sweep_finalize).
__global__ void __launch_bounds__(256) k_sweep_end(Dev *const *Dps, cudaGraphConditionalHandle h, int use_cond) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  const bool append = !st->stop && !st->stop_pending && st->search && !st->search_abort;
  sweep_finalize(D, st, append, h, use_cond);
}

// ---------------------------------------------------------------------------
// Sequential sweep (Alg. 5): the interfaces' steps one after another, each
// step's superblock built from the left set the previous step just extended.
// A step is the staged search with only interface k searching (k_seq_begin
// sets it), then k_seq_end: the cores are marked evaluated for the current
// ranks (the evaluation before this step covered them), the pivot appended at
// once, r_k raised; the last step of the sweep applies the stopping rules and
// counts the sweep.  The next step's new core slabs and the QR update of
// interface k follow in the ordinary kernels.
__global__ void k_seq_begin(Dev *const *Dps, int k) {
  if (threadIdx.x == 0) Dps[blockIdx.z]->st->seq_k = k;
}

__global__ void __launch_bounds__(256) k_seq_end(Dev *const *Dps, int k, int last) {
  const Dev &D = *Dps[blockIdx.z];
  State *st = D.st;
  const bool live = !st->stop && !st->stop_pending && st->search && k <= D.d - 1;
  if (live) sweep_append(D, st, k);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (live) {
      for (int q = 0; q <= D.d; ++q) st->ro[q] = st->r[q];
      IfaceState &I = st->it[k];
      st->search_evals += (long long)I.evals;
      if (I.active && I.accepted) { st->r[k] += 1; st->seq_nacc++; }
    }
    if (last) {
      if (st->stop) {
      } else if (st->stop_pending) {
        st->stop = 1;
        st->status = st->pending_status;
      } else if (!st->search) {
        st->sweep++;
      } else {
        if (st->rules && st->seq_nacc == 0) { st->stop = 1; st->status = ST_NO_PIVOT; }
        st->sweep++;
      }
      st->seq_k = 0;
      st->seq_nacc = 0;
    }
  }
}

// Serving: a warp per instance of the active set writes its stop flag, and
// for an instance that stopped its whole state, into (mapped) host memory;
// only_stopped_dd: rewrite just the states of the stopped double-double ones.
__global__ void __launch_bounds__(256) k_server_collect(Dev *const *Dps, int n, int *flags, State *states,
                                                        int only_stopped_dd) {
  const int q = blockIdx.x * TTQ_WARPS + warp_id(), lane = lane_id();
  if (q >= n) return;
  const Dev &D = *Dps[q];
  const State *st = D.st;
  const int stop = st->stop;
  if (!only_stopped_dd && lane == 0) flags[q] = stop;
  if (!stop || (only_stopped_dd && !D.prec)) return;
  static_assert(sizeof(State) % 8 == 0, "state copied in 8-byte words");
  const unsigned long long *src = reinterpret_cast<const unsigned long long *>(st);
  unsigned long long *dst = reinterpret_cast<unsigned long long *>(states + q);
  for (int i = lane; i < (int)(sizeof(State) / 8); i += 32) dst[i] = src[i];
}

// The tensor train of one instance copied out to a caller's buffer in the
// usual dense layouts: core k (1..d) as row-major r_{k-1} x N_k x r_k doubles
// (weights folded, no family constant), and for k = 1..d-1 the nested sets
// I<=k (r_k x k) and I>k (r_k x (d-k)) as row-major int32 node indices.
// Grid: x strides over the entries, y = k - 1.
struct TTExport {
  double *core[TTQ_MAXD + 1];
  int *left[TTQ_MAXD], *right[TTQ_MAXD];
  int r[TTQ_MAXD + 1];
};
__global__ void k_export_tt(Dev *const *Dps, int q, TTExport E) {
  const Dev &D = *Dps[q];
  const int k = blockIdx.y + 1, d = D.d;
  if (k > d) return;
  const int rl = E.r[k - 1], rr = E.r[k], N = D.N[k - 1];
  const long long n = (long long)rl * N * rr;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
  for (long long e = t0; e < n; e += nt) {
    const int b = (int)(e % rr), i = (int)((e / rr) % N), a = (int)(e / ((long long)rr * N));
    E.core[k][e] = D.Y[k][core_at(D, k, a, i, b)];
  }
  if (k <= d - 1) {
    for (long long e = t0; e < (long long)rr * k; e += nt) {
      const int a = (int)(e / k), m = (int)(e % k);
      E.left[k][e] = D.lidx[k][a * d + m];
    }
    for (long long e = t0; e < (long long)rr * (d - k); e += nt) {
      const int b = (int)(e / (d - k)), m = (int)(e % (d - k));
      E.right[k][e] = D.ridx[k][b * d + k + m];
    }
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
  pdl_wait();
  pdl_release();
  int running = 0;
  for (int q = threadIdx.x; q < count; q += blockDim.x) running |= !Dps[q]->st->stop;
  running = __syncthreads_or(running);
  if (threadIdx.x == 0) {
    const unsigned g = ++(*guard);
    cudaGraphSetConditional(h, (running && g < (unsigned)max_sweeps + 2) ? 1u : 0u);
  }
}

}  // namespace ttq
