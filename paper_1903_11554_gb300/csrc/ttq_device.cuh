// Device-side data layout and building blocks of the TT-cross quadrature.
//
// Layout of one plan in HBM (all inside the caller's workspace):
//   node tables   x[sum N], w[sum N], c[sum N] (2cosh s for the R^n form),
//                 T[N] = tanh^2(m h / 2) when every mode shares one uniform grid
//   index sets    per interface k = 1..d-1, capacity `cap` rows:
//                 lidx[k][a*d + m], m < k        node indices of I<=k (modes 1..k)
//                 ridx[k][b*d + m], m >= k       node indices of I>k  (modes k+1..d)
//                 lpar/lnode, rpar/rnode         parent-pointer form (Eq. 4)
//   cores         Y_k(alpha, i, beta) at ((beta * capL[k-1] + alpha) * N_k + i):
//                 the fiber matrix L_k = (r_{k-1} N_k) x r_k is column-major with
//                 leading dimension capL[k-1] * N_k, so a warp with lanes over
//                 the node index i reads and writes contiguous memory
//   node sums     V_k(alpha, beta) = sum_i Y_k(alpha, i, beta)  (+ double-double tail)
//   QR factors    of the cross matrix G_k = A(I<=k, I>k), r_k x r_k, ld = cap:
//                 Qr (row-major), Qc (col-major), Rc (col-major), Rr (row-major), 1/R_jj
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define TTQ_MAXD 32
#define TTQ_MAXR 128
#define TTQ_WARPS 8                      // warps per CTA in the fiber kernels
#define TTQ_CHUNK 128                    // at most this many nodes per piece of work of the rook kernels
#define TTQ_TIE_REL 1e-12                // Alg. 2 argmax: |E| >= max - (REL*max + ABS*scale) is a tie
#define TTQ_TIE_ABS 1e-14
#define TTQ_MAXPAIR 288                  // varying pairs of one cube-form fiber, <= (n/2)^2 for n <= 33
#define TTQ_MAX_INIT 1024                // initial random points scanned (include/ttq.h TTQ_MAX_INIT_SAMPLES)
#define TTQ_MAXP 4                       // pivots an interface may add per sweep (include/ttq.h TTQ_MAX_PIVOTS)

namespace ttq {

enum { FAM_C = 0, FAM_D = 1, FAM_E = 2, FAM_TEST = 3 };
enum { FORM_RN = 0, FORM_CUBE = 1 };

// status codes, mirror include/ttq.h
enum { ST_OK = 0, ST_NO_PIVOT = 1, ST_RANK_CAP = 2, ST_MAX_SWEEPS = 3,
       ST_ERR_NONFINITE = -2, ST_ERR_SINGULAR = -3, ST_ERR_TIMEOUT = -8 };

struct IfaceState {
  int active;          // a pivot search is running on this interface this sweep
  int rook_done;       // rook condition met
  int row, col;        // current rook position (rho, gamma)
  int rounds;
  int accepted;
  double err;          // residual at (row, col)
  unsigned long long evals;       // integrand evaluations of this sweep's search
  unsigned long long smax_bits;   // max score of the running stage's candidates (IEEE bits, >= 0)
  unsigned int stage_count;       // eligible candidates of the running stage
  int prow, prank;                // pvec holds R^-T L_k(prow, :)^T for the rank-prank factors (-1: none)
  unsigned items_done;            // work items of the running stage completed so far
  int fix[TTQ_MAXD];              // node indices the next rook step fixes: modes k.. of gamma
                                  // (column step), modes ..k-1 of rho (row step)
  unsigned epoch;                 // persistent search: stages of this sweep finished so far
  unsigned acc_arrive;            // several pivots per sweep: searches of the interface that ended (last decisions)
  int merged;                     // several pivots per sweep: stopped where it met an earlier search (its end
                                  // is that search's pivot)
};

struct State {
  int r[TTQ_MAXD + 1];      // current ranks, r[0] = r[d] = 1
  int ro[TTQ_MAXD + 1];     // ranks whose core entries are already evaluated
  int sweep;
  int status;               // ST_*
  int stop;                 // 1: the run is over; later kernels of the sweep do nothing
  int rules;                // 1: apply the stopping rules (full run); 0: stage calls
  int search;               // 1: run the pivot search this sweep
  int nonfinite;
  int singular;
  int nchanges;
  int stop_pending;         // a stopping rule fired in this sweep's contraction; applied at the end of the sweep
  int loop_guard;           // sweeps run by the device-side loop of this run (bounded by max_sweeps)
  int search_abort;         // persistent search: a wait passed its limit; every CTA leaves the search
  int seq_k;                // sequential sweep (Alg. 5): the interface whose step runs now (0: Alg. 6)
  int seq_nacc;             // sequential sweep: pivots accepted so far in this sweep
  unsigned batch_guard;     // sweeps run by a batch's loop (used in instance 0 of a batch)
  int pending_status;
  unsigned contract_arrive;  // CTAs of the two contraction chains that have finished
  unsigned end_arrive;      // CTAs of the last decisions kernel through the end of the sweep
  int qr_rank[TTQ_MAXD];    // size of the stored QR factors of G_k (0: none)
  int qr_row[TTQ_MAXD];     // rank whose row append is done (k_qr_row), 0: none pending
  unsigned long long scale_bits;   // max |core entry| as IEEE bits (non-negative)
  double value, value_lo, prev, conv;
  double changes[8];
  long long search_evals;
  long long init_evals;
  unsigned long long flops[16];    // algorithmic FP64 operations per kernel id (see ttq.cu)
  IfaceState it[TTQ_MAXD];
};

struct Dev {
  int d, family, form, n, cap, rook_max, init_samples, conv_window, max_sweeps, prec;
  int r0;                   // initial multi-indices (rank of every interface before the first sweep)
  unsigned long long wait_ns;   // persistent search: limit of every wait between CTAs (globaltimer ns)
  int uniformT;             // 1: D in R^n on one shared uniform grid -> pair table T
  int sblocks, cblocks, rblocks;   // CTAs: per interface (samples), per instance (column / row)
  int sms;                  // SMs of the device (placement of the item deals)
  int q_in_smem;            // the sample kernel stages Q_k in shared memory too (cap <= 96)
  double tol, pivot_tol, constant;
  unsigned long long seed;
  int N[TTQ_MAXD], off[TTQ_MAXD], S[TTQ_MAXD];
  int capL[TTQ_MAXD + 1];
  const double *x, *w, *c, *T;
  int *lidx[TTQ_MAXD], *ridx[TTQ_MAXD];
  int *lpar[TTQ_MAXD], *lnode[TTQ_MAXD], *rpar[TTQ_MAXD], *rnode[TTQ_MAXD];
  double *Y[TTQ_MAXD + 1];
  double *V[TTQ_MAXD + 1], *Vlo[TTQ_MAXD + 1];
  unsigned *vcnt[TTQ_MAXD + 1];   // per fiber: rows evaluated in this sweep
  double *Qr[TTQ_MAXD], *Qc[TTQ_MAXD], *Rc[TTQ_MAXD], *Rr[TTQ_MAXD], *rinv[TTQ_MAXD];
  double *Cc[TTQ_MAXD], *Sr[TTQ_MAXD];   // R D^-1 column-major, D^-1 R row-major (D = diag R)
  double *zvec[TTQ_MAXD];   // per interface: G^{-1} y or G^{-T} l of the next rook step
  double *pvec[TTQ_MAXD];   // per interface: R^{-T} l of the last row solve
  double *ptab[TTQ_MAXD];   // per interface: the next rook step's shared pair-factor product per node
  double *cbuf;             // the two contraction chains' vectors (hi, lo) x 2, cap each
  double *cs[TTQ_MAXD];     // per interface: scores |E| of the current candidates (-1: not eligible)
  double *ce[TTQ_MAXD];     // per interface: residuals E of the current candidates
  double *zs[TTQ_MAXD];     // per interface: z = G^-1 y of every random sample, cap apart
  double *im[TTQ_MAXD];     // per interface: max score of each row of 32 rook candidates (-1: none eligible)
  double *luh[TTQ_MAXD], *lul[TTQ_MAXD];   // double-double mode: P G_k = L U, column-major (hi, lo parts)
  int *lup[TTQ_MAXD];       // double-double mode: row i of P G_k is row lup[k][i] of G_k
  // several pivots per interface per sweep: npiv searches per interface; search
  // j's scratch lies j strides past search 0's (zvec: cap, ptab: pt_st, cs and
  // ce: cs_st, im: im_st entries) and its state is itx[(j - 1) TTQ_MAXD + k]
  int npiv, pt_st;
  size_t cs_st, im_st;
  IfaceState *itx;
  State *st;
};

// search j (0 .. npiv-1) of interface k: state and scratch
__device__ __forceinline__ IfaceState &search_state(const Dev &D, State *st, int k, int j) {
  return j == 0 ? st->it[k] : D.itx[(j - 1) * TTQ_MAXD + k];
}
__device__ __forceinline__ double *zvec_of(const Dev &D, int k, int j) { return D.zvec[k] + (size_t)j * D.cap; }
__device__ __forceinline__ double *ptab_of(const Dev &D, int k, int j) { return D.ptab[k] + (size_t)j * D.pt_st; }
__device__ __forceinline__ double *cs_of(const Dev &D, int k, int j) { return D.cs[k] + (size_t)j * D.cs_st; }
__device__ __forceinline__ double *ce_of(const Dev &D, int k, int j) { return D.ce[k] + (size_t)j * D.cs_st; }
__device__ __forceinline__ double *im_of(const Dev &D, int k, int j) { return D.im[k] + (size_t)j * D.im_st; }

// ---------------------------------------------------------------------------
// warp helpers (fixed butterfly order: every lane gets the same, reproducible result)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_prod(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// argmax with ties to the lowest index; score -1 marks "no candidate"
struct Best {
  double score;
  int idx;
  double val;
};
__device__ __forceinline__ bool better(double s1, int i1, double s2, int i2) {
  return s1 > s2 || (s1 == s2 && i1 < i2);
}
__device__ __forceinline__ Best warp_best(Best b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double s = __shfl_xor_sync(0xffffffffu, b.score, o);
    int i = __shfl_xor_sync(0xffffffffu, b.idx, o);
    double v = __shfl_xor_sync(0xffffffffu, b.val, o);
    if (better(s, i, b.score, b.idx)) { b.score = s; b.idx = i; b.val = v; }
  }
  return b;
}

// ---------------------------------------------------------------------------
// double-double arithmetic (Dekker 1971; Knuth's TwoSum; TwoProd through FMA)

struct dd { double hi, lo; };
__device__ __forceinline__ dd two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dd fast_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
  double p = a.hi * b;
  double e = fma(a.hi, b, -p);
  e = fma(a.lo, b, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  double p = a.hi * b.hi;
  double e = fma(a.hi, b.hi, -p);
  e = fma(a.hi, b.lo, e);
  e = fma(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dd dd_div_d(dd a, double b) {
  double q1 = a.hi / b;
  dd p = {q1 * b, fma(q1, b, -(q1 * b))};      // q1*b exactly
  dd r = dd_add(a, {-p.hi, -p.lo});
  double q2 = r.hi / b;
  return fast_two_sum(q1, q2);
}
// a / b for double-double b: three quotient digits by the leading part of b,
// each followed by the exact remainder (long division, Dekker 1971)
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  const double q1 = a.hi / b.hi;
  dd r = dd_add(a, dd_mul({-b.hi, -b.lo}, {q1, 0.0}));
  const double q2 = r.hi / b.hi;
  r = dd_add(r, dd_mul({-b.hi, -b.lo}, {q2, 0.0}));
  const double q3 = r.hi / b.hi;
  dd q = fast_two_sum(q1, q2);
  return dd_add(q, {q3, 0.0});
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd warp_sum_dd(dd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd u = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    // combine in a lane-order-independent way: lower lane's value first
    int lane = threadIdx.x & 31;
    v = ((lane & o) == 0) ? dd_add(v, u) : dd_add(u, v);
  }
  return v;
}

// ---------------------------------------------------------------------------
// 1/x for the R^n integrands' (sum 2 cosh s)^-2, x >= 2: the hardware's
// approximate reciprocal (PTX rcp.approx.ftz.f64) refined by two Newton-Raphson
// steps y <- y + y (1 - x y), each of which squares the relative error, so the
// result is within an ulp of 1/x in four multiply-adds instead of a full IEEE
// division (FP64 instructions are the kernels' scarce resource here).
__device__ __forceinline__ double recip_nr(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// SplitMix64 (Steele, Lea & Flood 2014): m-th output from state s is mix(s + m*GAMMA)

__device__ __forceinline__ unsigned long long sm_mix(unsigned long long z) {
  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ULL;
  z ^= z >> 27; z *= 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long sm_out(unsigned long long s, unsigned long long m) {
  return sm_mix(s + m * 0x9E3779B97F4A7C15ULL);
}
__device__ __forceinline__ unsigned long long stream_id(int sweep, int k, int purpose) {
  return ((unsigned long long)(unsigned)sweep << 32) | ((unsigned long long)(k & 0xFFFFFF) << 8) |
         (unsigned long long)(purpose & 0xFF);
}
__device__ __forceinline__ int draw_index(unsigned long long seed, unsigned long long stream,
                                          unsigned long long counter, unsigned long long M) {
  unsigned long long s1 = sm_out(seed, 1);
  unsigned long long s2 = sm_out(s1, stream + 1);
  unsigned long long v = sm_out(s2, counter + 1);
  return (int)__umul64hi(v, M);
}

// Slot of a warp in a round-robin deal of work items over a grid that fills the
// device's resident CTA slots (CTA c on SM c mod sms in the first wave).  Items
// w = slot * gridDim.x + blockIdx.x; with `per` items per CTA the CTAs sharing an
// SM rotate their slots by per each, so their items continue one deal over the
// SM's four schedulers (FP64 issue is per scheduler) instead of all starting at
// warp 0.
__device__ __forceinline__ int deal_slot(int warp, int sms, long long total) {
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  const int rot = (int)(((long long)(blockIdx.x / (sms > 0 ? sms : gridDim.x)) * per) & 7);
  return (warp - rot) & 7;
}

// The instance's descriptor copied to shared memory by the whole CTA (one
// round of parallel loads) before anything else: it never changes during a
// run, so the copy may overlap the previous kernel (it precedes pdl_wait), and
// afterwards every descriptor field is a shared-memory read instead of the
// first link of a chain of dependent global loads.
__device__ __forceinline__ const Dev &stage_dev(Dev *const *Dps, Dev &sD) {
  static_assert(sizeof(Dev) % 8 == 0, "descriptor copied in 8-byte words");
  const unsigned long long *src = reinterpret_cast<const unsigned long long *>(Dps[blockIdx.z]);
  unsigned long long *dst = reinterpret_cast<unsigned long long *>(&sD);
  for (int i = threadIdx.x; i < (int)(sizeof(Dev) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  return sD;
}

// Programmatic dependent launch: pdl_wait blocks until the preceding kernel of
// the stream has completed and its writes are visible; pdl_release lets the
// next kernel begin launching.  Both are no-ops for a kernel launched without
// the programmatic-serialization attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;\n" :::); }

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// Fiber evaluation (kernel (a)'s core routine).
//
// One warp evaluates the weighted tensor A at the points that share every node
// index except the free mode f: (m_0, .., m_{f-1}, i, m_{f+1}, .., m_{d-1}) for a
// range of i.  The factors that do not involve mode f (the weights and node
// terms of the other modes, and for D / E every pair of other modes) are the
// same for the whole fiber; the warp computes them once, cooperatively (lanes
// split the modes and pairs, butterfly reductions combine them), and each lane
// then adds only the factors that involve its own node i.  Every entry is still
// exactly the integrand at that point, up to rounding.

struct FiberU {
  double W;       // prod of weights of the other modes
  double WP;      // R^n: W times P
  double S;       // R^n: sum 2cosh s of other modes; TEST: sum of x
  double P;       // product of the pair factors among the other modes
  double aL, bL, aR, bR;   // unit-cube B_n: left/right sums as a + b * x_F
  int npair;      // unit-cube A_n: number of pairs (i, j) whose product contains x_F
  int fl_node;    // FP64 operations per node of this fiber (the lane-local part)
  int fl_uniform; // FP64 operations of the fiber's shared part
  const double *T;  // D in R^n on one uniform grid: the pair table (the CTA's shared copy, else D.T)
};

// The pair table T of D in R^n on one uniform grid copied to the CTA's shared
// memory (dyn: the launch's dynamic shared memory); null when the problem has
// none or the launch gave it less than N doubles.  Constant for the plan, so it is copied before the
// kernel's wait; the caller's barrier orders the copy before its reads.
__device__ __forceinline__ const double *stage_pair_table(const Dev &D, double *dyn) {
  unsigned bytes;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(bytes));
  if (!D.uniformT || D.N[0] > (int)(bytes / 8)) return nullptr;
  for (int t = threadIdx.x; t < D.N[0]; t += blockDim.x) dyn[t] = D.T[t];
  return dyn;
}

// q-th pair (a, b), a < b, of d modes in row order: the row from the
// triangular-number inverse a = d - 2 - floor((sqrt(4 d (d-1) - 7 - 8 q) - 1) / 2)
// (an FP32 square root of an integer below 4000, exact for every q of every
// d <= 32), the column from the row's first index; a loop over the rows would
// cost up to d - 1 dependent steps per pair
__device__ __forceinline__ void pair_of(int q, int d, int &a, int &b) {
  const float sq = sqrtf((float)(4 * d * (d - 1) - 7 - 8 * q));
  a = d - 2 - (int)floorf((sq - 1.0f) * 0.5f);
  b = q + a + 1 - d * (d - 1) / 2 + (d - a) * (d - a - 1) / 2;
}

// m: warp-uniform node indices (shared memory); plist: per-warp scratch of TTQ_MAXPAIR doubles;
// Ts: the CTA's shared-memory copy of the pair table T, or null (T read from global memory)
__device__ __forceinline__ FiberU fiber_setup(const Dev &D, int f, const int *m, double *plist,
                                              const double *Ts = nullptr) {
  const int lane = threadIdx.x & 31;
  const int d = D.d;
  FiberU u;
  u.P = 1.0; u.S = 0.0; u.aL = u.bL = u.aR = u.bR = 0.0; u.npair = 0;
  u.T = Ts ? Ts : D.T;
  const double *T = u.T;
  double wj = 1.0;
  const bool mine = lane < d && lane != f;
  const int oj = mine ? D.off[lane] + m[lane] : 0;
  if (mine) wj = D.w[oj];
  // R^n: this lane's 2 cosh s and, for D on a uniform grid, its first pair
  // factors are loaded with the weight, before the reductions, so the loads of
  // the shared part overlap instead of following each other
  double cj = 0.0, tp[3] = {1.0, 1.0, 1.0};
  const bool rn_pairs = D.form == FORM_RN && D.family == FAM_D && D.uniformT;
  if (D.form == FORM_RN && D.family != FAM_TEST && mine) cj = D.c[oj];
  if (rn_pairs) {
    const int np = d * (d - 1) / 2;
#pragma unroll
    for (int qq = 0; qq < 3; ++qq) {
      const int q = lane + 32 * qq;
      if (q < np) {
        int a, b;
        pair_of(q, d, a, b);
        if (a != f && b != f) {
          const int dm = m[a] - m[b];
          tp[qq] = T[dm < 0 ? -dm : dm];
        }
      }
    }
  }
  u.W = warp_prod(wj);
  u.WP = u.W;
  u.fl_uniform = d - 1;
  if (D.family == FAM_TEST) {
    double xj = (lane < d && lane != f) ? D.x[D.off[lane] + m[lane]] : 0.0;
    u.S = warp_sum(xj);
    u.fl_uniform += d - 1;
    u.fl_node = 2 * D.n + 5;
    return u;
  }
  if (D.form == FORM_RN) {
    u.S = warp_sum(cj);
    u.fl_uniform += d - 1;
    u.fl_node = 13;                             // add, reciprocal (1 + 8), square, 2 products
    if (D.family == FAM_D) {
      u.fl_node += d - 1;                       // the pair factors with the free mode
      u.fl_uniform += (d - 1) * (d - 2) / 2 * (D.uniformT ? 1 : 4);
      // the pairs of other modes dealt over the lanes: one FP64 product per 32
      // pairs on the warp's instruction stream instead of d - 1 on lane 0's
      double p = 1.0;
      const int np = d * (d - 1) / 2;
      int q0 = lane;
      if (rn_pairs) {                         // the first three were loaded above
        p = (tp[0] * tp[1]) * tp[2];
        q0 = lane + 96;
      }
      for (int q = q0; q < np; q += 32) {
        int a, b;
        pair_of(q, d, a, b);
        if (a == f || b == f) continue;
        double t2;
        if (D.uniformT) {
          int dm = m[a] - m[b];
          t2 = T[dm < 0 ? -dm : dm];
        } else {
          double t = tanh((D.x[D.off[a] + m[a]] - D.x[D.off[b] + m[b]]) * 0.5);
          t2 = t * t;
        }
        p *= t2;
      }
      u.P = warp_prod(p);
      u.WP = u.W * u.P;
    }
    return u;
  }
  // unit cube: variable x_v (v = 2..n) lives in mode v-2; free variable F = f + 2
  const int n = D.n, F = f + 2;
#define XV(v) (D.x[D.off[(v) - 2] + m[(v) - 2]])
  if (D.family == FAM_C || D.family == FAM_D) {
    if (lane == 0) {
      double p = 1.0, aL = 1.0;
      for (int v = 2; v <= F - 1; ++v) { p *= XV(v); aL += p; }
      double PL = p, t = 1.0;
      p = 1.0;
      for (int v = F + 1; v <= n; ++v) { p *= XV(v); t += p; }
      double aR = 1.0;
      p = 1.0;
      for (int v = n; v >= F + 1; --v) { p *= XV(v); aR += p; }
      double PR = p, h = 1.0;
      p = 1.0;
      for (int v = F - 1; v >= 2; --v) { p *= XV(v); h += p; }
      u.aL = aL; u.bL = PL * t; u.aR = aR; u.bR = PR * h;
    }
    u.fl_uniform += 4 * n;
    u.fl_node = 8;
    u.aL = __shfl_sync(0xffffffffu, u.aL, 0);
    u.bL = __shfl_sync(0xffffffffu, u.bL, 0);
    u.aR = __shfl_sync(0xffffffffu, u.aR, 0);
    u.bR = __shfl_sync(0xffffffffu, u.bR, 0);
  }
  if (D.family == FAM_D || D.family == FAM_E) {
    // pairs 1 <= i < j <= n with p_ij = x_{i+1} ... x_j; lane handles row i = lane + 1
    double pu = 1.0;
    const int i = lane + 1;
    const int width = n - F + 1;
    if (i <= n - 1) {
      double p = 1.0;
      for (int j = i + 1; j <= n; ++j) {
        if (j != F) p *= XV(j);
        if (i < F && F <= j) {
          plist[(i - 1) * width + (j - F)] = p;        // x_F * p is this pair's product
        } else {
          double q = (1.0 - p) / (1.0 + p);
          pu *= q * q;
        }
      }
    }
    u.P = warp_prod(pu);
    u.npair = (F - 1) * width;
    u.fl_uniform += 6 * (n * (n - 1) / 2 - u.npair);
    u.fl_node = (D.family == FAM_D ? 11 : 5) + 6 * u.npair;
    __syncwarp();
  }
#undef XV
  return u;
}

// The same value for the R^n form of D on one uniform grid when the pair
// factors of the free mode with the modes outside [jlo, jhi) are the same for
// every fiber of the step and their product per node sits in tab (built once
// per rook step): tab[i] * prod_{jlo <= j < jhi, j != f} T(i, m_j) replaces the
// product over all d - 1 other modes.
__device__ __forceinline__ double fiber_value_tab(const Dev &D, int f, const int *m, const FiberU &u,
                                                  int i, const double *tab, int jlo, int jhi) {
  const int o = D.off[f] + i;
  const double wi = D.w[o];
  const double s = u.S + D.c[o];
  const double rs = recip_nr(s);
  double p = u.WP * wi * __ldcg(tab + i);         // rebuilt every rook step: read through L2
  for (int j = jlo; j < jhi; ++j) {
    if (j == f) continue;
    const int dm = i - m[j];
    p *= u.T[dm < 0 ? -dm : dm];
  }
  return p * (rs * rs);
}

// value at node i of the free mode f (lane-local)
__device__ __forceinline__ double fiber_value(const Dev &D, int f, const int *m, const FiberU &u,
                                              const double *plist, int i) {
  const int o = D.off[f] + i;
  const double wi = D.w[o];
  if (D.family == FAM_TEST) {
    double e = exp(-(u.S + D.x[o]) / (double)D.d);
    double g = 0.0;
    for (int t = 0; t < D.n; ++t) g = (g + 1.0) * e;
    return u.W * wi * g;
  }
  if (D.form == FORM_RN) {
    // W P w_i prod_j T(i, m_j) / s^2 with W P the fiber's shared product
    const double s = u.S + D.c[o];
    const double rs = recip_nr(s);
    double p = u.WP * wi;
    if (D.family == FAM_D) {
      const int d = D.d;
      if (D.uniformT) {
        for (int j = 0; j < d; ++j) {
          if (j == f) continue;
          int dm = i - m[j];
          p *= u.T[dm < 0 ? -dm : dm];
        }
      } else {
        const double si = D.x[o];
        for (int j = 0; j < d; ++j) {
          if (j == f) continue;
          double t = tanh((si - D.x[D.off[j] + m[j]]) * 0.5);
          p *= t * t;
        }
      }
    }
    return p * (rs * rs);
  }
  const double xf = D.x[o];
  double g = 1.0;
  if (D.family == FAM_D || D.family == FAM_E) {
    double num = 1.0, den = 1.0;
    for (int t = 0; t < u.npair; ++t) {
      double cx = plist[t];
      num *= fma(-xf, cx, 1.0);
      den *= fma(xf, cx, 1.0);
    }
    double q = num / den;
    g = u.P * q * q;
  }
  if (D.family == FAM_C || D.family == FAM_D) {
    g = g / ((u.aL + u.bL * xf) * (u.aR + u.bR * xf));
  }
  return u.W * wi * g;
}

// ---------------------------------------------------------------------------
// Single-point evaluation (one thread): A(m) = prod_v w_{m_v} g(x_{m_0}, .., x_{m_{d-1}})
// for the node indices m_v = m[v * stride].  The same integrand as the fiber
// routines above, for work where every thread holds its own point.

__device__ __forceinline__ double point_value(const Dev &D, const int *m, int stride) {
  const int d = D.d;
  double W = 1.0;
  for (int v = 0; v < d; ++v) W *= D.w[D.off[v] + m[v * stride]];
  if (D.family == FAM_TEST) {
    double S = 0.0;
    for (int v = 0; v < d; ++v) S += D.x[D.off[v] + m[v * stride]];
    const double e = exp(-S / (double)d);
    double g = 0.0;
    for (int t = 0; t < D.n; ++t) g = (g + 1.0) * e;
    return W * g;
  }
  if (D.form == FORM_RN) {
    double s = 0.0;
    for (int v = 0; v < d; ++v) s += D.c[D.off[v] + m[v * stride]];
    const double rs = recip_nr(s);
    double g = rs * rs;
    if (D.family == FAM_D) {
      double p = 1.0;
      for (int a = 0; a < d; ++a) {
        const int ma = m[a * stride];
        for (int b = a + 1; b < d; ++b) {
          const int mb = m[b * stride];
          if (D.uniformT) {
            const int dm = ma - mb;
            p *= D.T[dm < 0 ? -dm : dm];
          } else {
            const double t = tanh((D.x[D.off[a] + ma] - D.x[D.off[b] + mb]) * 0.5);
            p *= t * t;
          }
        }
      }
      g *= p;
    }
    return W * g;
  }
  // unit cube: variable x_v (v = 2..n) lives in mode v-2
  const int n = D.n;
#define XP(v) (D.x[D.off[(v) - 2] + m[((v) - 2) * stride]])
  double g = 1.0;
  if (D.family == FAM_D || D.family == FAM_E) {
    // A_n: pairs 1 <= i < j <= n with p_ij = x_{i+1} ... x_j, q = (1 - p) / (1 + p)
    double num = 1.0, den = 1.0;
    for (int i = 1; i <= n - 1; ++i) {
      double p = 1.0;
      for (int j = i + 1; j <= n; ++j) {
        p *= XP(j);
        num *= 1.0 - p;
        den *= 1.0 + p;
      }
    }
    const double q = num / den;
    g = q * q;
  }
  if (D.family == FAM_C || D.family == FAM_D) {
    double left = 1.0, right = 1.0, p = 1.0;
    for (int v = 2; v <= n; ++v) { p *= XP(v); left += p; }
    p = 1.0;
    for (int v = n; v >= 2; --v) { p *= XP(v); right += p; }
    g = g / (left * right);
  }
#undef XP
  return W * g;
}

// The same value, evaluated by a group of G lanes (lanes gl = 0..G-1 of an
// aligned group, G a power of two <= 32): modes, pairs and rows of the
// unit-cube pair product are dealt over the group and combined by butterflies
// within it; every lane of the group returns A.  A lane's share of the FP64
// instructions is ~1/G of a single lane's.
template <int G>
__device__ __forceinline__ double group_prod(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int G>
__device__ __forceinline__ double group_point_value(const Dev &D, const int *m, int stride, int gl) {
  const int d = D.d;
  // a lane's modes (at most 32 / G of them): their weights and, for R^n, 2 cosh s
  // loaded together before any product, so the loads overlap
  constexpr int MV = (TTQ_MAXD + G - 1) / G;
  double wv[MV], cv[MV];
  const bool rn = D.form == FORM_RN && D.family != FAM_TEST;
#pragma unroll
  for (int u = 0; u < MV; ++u) {
    const int v = gl + u * G;
    const int o = v < d ? D.off[v] + m[v * stride] : 0;
    wv[u] = v < d ? D.w[o] : 1.0;
    cv[u] = (v < d && rn) ? D.c[o] : 0.0;
  }
  double W = 1.0;
#pragma unroll
  for (int u = 0; u < MV; ++u) W *= wv[u];
  W = group_prod<G>(W);
  if (D.family == FAM_TEST) {
    double S = 0.0;
    for (int v = gl; v < d; v += G) S += D.x[D.off[v] + m[v * stride]];
    S = group_sum<G>(S);
    const double e = exp(-S / (double)d);
    double g = 0.0;
    for (int t = 0; t < D.n; ++t) g = (g + 1.0) * e;
    return W * g;
  }
  if (D.form == FORM_RN) {
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < MV; ++u) s += cv[u];
    s = group_sum<G>(s);
    const double rs = recip_nr(s);
    double g = rs * rs;
    if (D.family == FAM_D) {
      double p = 1.0;
      const int np = d * (d - 1) / 2;
      if (D.uniformT) {
        for (int q0 = gl; q0 < np; q0 += 4 * G) {   // four pair factors' loads in flight
          double t4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * G;
            t4[u] = 1.0;
            if (q < np) {
              int a, b;
              pair_of(q, d, a, b);
              const int dm = m[a * stride] - m[b * stride];
              t4[u] = D.T[dm < 0 ? -dm : dm];
            }
          }
          p *= (t4[0] * t4[1]) * (t4[2] * t4[3]);
        }
      } else {
        for (int q = gl; q < np; q += G) {
          int a, b;
          pair_of(q, d, a, b);
          const int ma = m[a * stride], mb = m[b * stride];
          const double t = tanh((D.x[D.off[a] + ma] - D.x[D.off[b] + mb]) * 0.5);
          p *= t * t;
        }
      }
      g *= group_prod<G>(p);
    }
    return W * g;
  }
  const int n = D.n;
#define XG(v) (D.x[D.off[(v) - 2] + m[((v) - 2) * stride]])
  double g = 1.0;
  if (D.family == FAM_D || D.family == FAM_E) {
    // A_n: rows i of the pair product dealt over the group
    double num = 1.0, den = 1.0;
    for (int i = 1 + gl; i <= n - 1; i += G) {
      double p = 1.0;
      for (int j = i + 1; j <= n; ++j) {
        p *= XG(j);
        num *= 1.0 - p;
        den *= 1.0 + p;
      }
    }
    num = group_prod<G>(num);
    den = group_prod<G>(den);
    const double q = num / den;
    g = q * q;
  }
  if (D.family == FAM_C || D.family == FAM_D) {
    double left = 1.0, right = 1.0, p = 1.0;
    for (int v = 2; v <= n; ++v) { p *= XG(v); left += p; }
    p = 1.0;
    for (int v = n; v >= 2; --v) { p *= XG(v); right += p; }
    g = g / (left * right);
  }
#undef XG
  return W * g;
}

// FP64 operations of one point_value (algorithmic count)
__device__ __forceinline__ int point_flops(const Dev &D) {
  const int d = D.d, n = D.n;
  if (D.family == FAM_TEST) return 2 * (d - 1) + 2 * n + 3;
  if (D.form == FORM_RN) return 2 * (d - 1) + 13 + (D.family == FAM_D ? d * (d - 1) / 2 * (D.uniformT ? 1 : 4) + 1 : 0);
  int fl = d;
  if (D.family == FAM_D || D.family == FAM_E) fl += 3 * n * (n - 1) / 2 + 2;
  if (D.family == FAM_C || D.family == FAM_D) fl += 4 * n + 2;
  return fl;
}

}  // namespace ttq
