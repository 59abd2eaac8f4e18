// libttq: C ABI of the GB300 TT-cross quadrature (declarations and contracts in include/ttq.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <string>
#include <vector>
#include <mutex>

#include "../../include/ttq.h"
#include "ttq_kernels.cuh"

using namespace ttq;

static thread_local std::string g_last_error;

static int set_err(int code, const char *msg) {
  g_last_error = msg;
  return code;
}

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      g_last_error = std::string(#call) + ": " + cudaGetErrorString(e_);           \
      return TTQ_ERR_CUDA;                                                         \
    }                                                                              \
  } while (0)

// kernel ids of the timing counters (ttq_plan_kernel_times)
enum { KT_EVAL = 0, KT_QR, KT_CONTRACT, KT_SAMPLES, KT_ROOK_COL, KT_ROOK_ROW, KT_UPDATE, KT_INIT, KT_SETUP,
       KT_SOLVE, KT_SEARCH, KT_N };

#define TTQ_RESULT_SLOTS 64

struct TimedLaunch {
  int kid;
  cudaEvent_t a, b;
};

// A plan is a set of `count` instances (one integral each) that share every
// kernel launch: instance q is blockIdx.z == q.  A single-integral plan is a
// set of one; a batch is a set of many with uneven d, N and rank caps.
struct ttq_plan {
  int count;
  Dev h;                    // host copy of instance 0's descriptor
  Dev *dev;                 // instance 0's descriptor (device)
  State *st;                // instance 0's state (device)
  Dev **devs;               // device array of every instance's descriptor
  Dev *hs;                  // host copies of every descriptor (&h when count == 1)
  State **sts;              // every instance's state, device (&st when count == 1)
  unsigned *guard;          // device loop counter of a batch's WHILE node
  cudaStream_t stream;
  // launch configuration (batch maxima)
  int max_ni, rook_max, max_sweeps, max_cap;
  int grid_eval, sblocks, cblocks, rblocks, max_sum_n;
  int qr_smem, samples_smem, contract_smem, solve_smem;
  int tsm_smem;             // kernel (a): room for the pair table of D in R^n (N doubles)
  long long launches;
  State *hst;               // pinned host mirror of the states (count entries)
  int timing;               // 1: bracket every launch with CUDA events
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> pool;
  double kt_ms[KT_N];
  long long kt_n[KT_N];
  long long h2d, d2h;       // bytes copied host<->device by this plan
  cudaStream_t s2;          // side stream: the contraction runs beside the pivot search
  cudaEvent_t fork, join;
  int use_graph;            // whole run as one graph (timing off, not the legacy stream)
  cudaGraphExec_t sweep_exec;
  cudaGraphExec_t run_exec; // WHILE(any instance running) { one sweep }
  cudaGraphConditionalHandle cond;
  int in_loop;              // enqueueing the body of the WHILE node
  int sweep_kernels;        // kernels in one sweep
  State *slots;             // pinned host copies of the final state of launched runs
  int sequential;           // sweeps of Alg. 5 (interfaces one after another) instead of Alg. 6
  int persistent;           // one instance: the search of a sweep as one cooperative launch (k_search)
  int search_grid, search_smem;
  int npiv;                 // searches per interface (several pivots per sweep): the decisions kernels' grid y
  int rook_rmax;            // largest rook work item, rows of 32 candidates (1, 2 or 4)
  // batches: the instances sorted by cost (rank cap^2 x nodes), split into
  // ngroups contiguous groups that run as concurrent WHILE loops of one graph
  Dev **devs_sorted;        // device array, count entries, in cost order
  int ngroups;
  std::vector<int> order;   // instance of each sorted position
  std::vector<int> glo, gcnt, gkernels;   // per group: first sorted position, instances, kernels per iteration
  // the group being enqueued (the whole batch when cur_dv is null)
  Dev *const *cur_dv;
  int cur_nb;
  unsigned *cur_guard;
};

static cudaEvent_t ev_get(ttq_plan *P) {
  if (!P->pool.empty()) {
    cudaEvent_t e = P->pool.back();
    P->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// The second stream (QR row append, contraction).  For one instance it runs
// at the device's highest priority and graphs are instantiated with their
// nodes' priorities: at the start of a graph body the QR row kernel's 11-odd
// CTAs are dispatched before kernel (a)'s instead of waiting behind them.  For
// a batch (hundreds of CTAs on the second stream, off the critical path) it
// keeps the default priority.
static cudaError_t create_side_stream(cudaStream_t *s2, bool high) {
  if (!high) return cudaStreamCreateWithFlags(s2, cudaStreamNonBlocking);
  int lo = 0, hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (e != cudaSuccess) return e;
  return cudaStreamCreateWithPriority(s2, cudaStreamNonBlocking, hi);
}

// launch helper: counts the launch and, when timing, records events around it
// Kernel launch in the sweep chain: with programmatic serialization (the next
// kernel launches while this one drains; its pdl_wait orders the data), except
// while per-kernel timing is on.
template <typename... KArgs, typename... Args>
static void launch_k(ttq_plan *P, void (*kern)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s,
                     Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = P->timing ? 0 : 1;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename F>
static void timed_on(ttq_plan *P, cudaStream_t s, int kid, F &&launch) {
  if (P->timing) {
    TimedLaunch t{kid, ev_get(P), ev_get(P)};
    cudaEventRecord(t.a, s);
    launch();
    cudaEventRecord(t.b, s);
    P->pending.push_back(t);
  } else {
    launch();
  }
  P->launches++;
  P->kt_n[kid]++;
}
template <typename F>
static void timed(ttq_plan *P, int kid, F &&launch) {
  timed_on(P, P->stream, kid, launch);
}

// fold the completed launches' durations into the counters (stream must be idle)
static void harvest(ttq_plan *P) {
  for (auto &t : P->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) P->kt_ms[t.kid] += ms;
    P->pool.push_back(t.a);
    P->pool.push_back(t.b);
  }
  P->pending.clear();
}

// ---------------------------------------------------------------------------
// validation and layout

static int validate(const ttq_problem *p) {
  if (!p) return set_err(TTQ_ERR_INVALID_ARG, "null problem");
  if (p->family < 0 || p->family > 3) return set_err(TTQ_ERR_INVALID_ARG, "bad family");
  if (p->form < 0 || p->form > 1) return set_err(TTQ_ERR_INVALID_ARG, "bad form");
  if (p->d < 2 || p->d > TTQ_MAX_MODES) return set_err(TTQ_ERR_INVALID_ARG, "d must be in 2..32");
  if (p->family == TTQ_FAMILY_TEST) {
    if (p->n < 1) return set_err(TTQ_ERR_INVALID_ARG, "TEST needs n >= 1 terms");
  } else if (p->form == TTQ_FORM_RN) {
    if (p->family == TTQ_FAMILY_E) return set_err(TTQ_ERR_INVALID_ARG, "E_n has no R^n form");
    if (p->d != p->n) return set_err(TTQ_ERR_INVALID_ARG, "R^n form needs d == n");
  } else if (p->d != p->n - 1) {
    return set_err(TTQ_ERR_INVALID_ARG, "unit-cube form needs d == n - 1");
  }
  if (!p->nodes_per_mode || !p->nodes || !p->weights) return set_err(TTQ_ERR_INVALID_ARG, "null arrays");
  for (int k = 0; k < p->d; ++k)
    if (p->nodes_per_mode[k] < 2 || p->nodes_per_mode[k] > TTQ_MAX_NODES)
      return set_err(TTQ_ERR_INVALID_ARG, "N_k must be in 2..2048");
  if (p->rank_cap < 1 || p->rank_cap > TTQ_MAX_RANK) return set_err(TTQ_ERR_INVALID_ARG, "rank_cap must be in 1..128");
  if (!(p->tol >= 0.0) || !(p->pivot_tol >= 0.0)) return set_err(TTQ_ERR_INVALID_ARG, "negative tolerance");
  if (p->conv_window < 1 || p->conv_window > 8) return set_err(TTQ_ERR_INVALID_ARG, "conv_window must be in 1..8");
  if (p->max_sweeps < 1) return set_err(TTQ_ERR_INVALID_ARG, "max_sweeps must be >= 1");
  if (p->rook_max < 1) return set_err(TTQ_ERR_INVALID_ARG, "rook_max must be >= 1");
  if (p->init_samples < 1 || p->init_samples > TTQ_MAX_INIT_SAMPLES)
    return set_err(TTQ_ERR_INVALID_ARG, "init_samples must be in 1..1024");
  {
    const int r0 = p->r0 < 1 ? 1 : p->r0;
    if (p->r0 < 0 || r0 > p->rank_cap || r0 > p->init_samples || r0 > p->nodes_per_mode[0] ||
        r0 > p->nodes_per_mode[p->d - 1])
      return set_err(TTQ_ERR_INVALID_ARG, "r0 must be in 1..min(rank_cap, init_samples, N_1, N_d)");
  }
  if (p->n_samples < 0 || p->n_samples > (1 << 20)) return set_err(TTQ_ERR_INVALID_ARG, "bad n_samples");
  if (p->precision < 0 || p->precision > 1) return set_err(TTQ_ERR_INVALID_ARG, "bad precision");
  if (p->npiv < 0 || p->npiv > TTQ_MAX_PIVOTS) return set_err(TTQ_ERR_INVALID_ARG, "npiv must be in 0..4");
  return TTQ_OK;
}

static int npiv_of(const ttq_problem *p) { return p->npiv < 1 ? 1 : p->npiv; }

// a batch's workspace head: its descriptor array, then the same sorted by cost
static size_t batch_head_bytes(int count) {
  return count > 1 ? 2 * (((size_t)count * sizeof(Dev *) + 255) & ~(size_t)255) : 0;
}

// cost of an instance for the grouping of a batch: rank cap^2 x nodes
static double instance_cost(const ttq_problem *p) {
  double n = 0.0;
  for (int k = 0; k < p->d; ++k) n += p->nodes_per_mode[k];
  return (double)p->rank_cap * p->rank_cap * n;
}

struct Bump {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = (off + 255) & ~(size_t)255;
    off = o + bytes;
    return o;
  }
};

struct Layout {
  size_t dev, st, x, w, c, T, cbuf;
  size_t lidx[TTQ_MAXD], ridx[TTQ_MAXD], lpar[TTQ_MAXD], lnode[TTQ_MAXD], rpar[TTQ_MAXD], rnode[TTQ_MAXD];
  size_t Y[TTQ_MAXD + 1], V[TTQ_MAXD + 1], Vlo[TTQ_MAXD + 1];
  size_t vcnt[TTQ_MAXD + 1], vcnt_all, vcnt_bytes;   // fiber row counters: one region, zeroed at creation
  size_t Qr[TTQ_MAXD], Qc[TTQ_MAXD], Rc[TTQ_MAXD], Rr[TTQ_MAXD], Cc[TTQ_MAXD], Sr[TTQ_MAXD], rinv[TTQ_MAXD],
      zvec[TTQ_MAXD], pvec[TTQ_MAXD], ptab[TTQ_MAXD];
  size_t cs[TTQ_MAXD], ce[TTQ_MAXD], im[TTQ_MAXD], zs[TTQ_MAXD];
  size_t itx;                // states of searches 1 .. npiv-1 (several pivots per sweep)
  size_t cs_st, im_st;       // scratch strides between the searches of an interface
  int pt_st;
  size_t luh[TTQ_MAXD], lul[TTQ_MAXD], lup[TTQ_MAXD];   // double-double LU of G_k (precision DD only)
  size_t devs;               // this instance's own one-entry descriptor array
  size_t total;
  int sblocks, cblocks, rblocks;
};

static int samples_for(const ttq_problem *p, int k) {  // interface k = 1..d-1
  return p->n_samples > 0 ? p->n_samples : p->nodes_per_mode[k - 1] + p->nodes_per_mode[k];
}

static void make_layout(const ttq_problem *p, Layout *L) {
  const int d = p->d, cap = p->rank_cap;
  size_t sumN = 0;
  int maxN = 0, maxS = 0;
  for (int k = 0; k < d; ++k) { sumN += p->nodes_per_mode[k]; maxN = p->nodes_per_mode[k] > maxN ? p->nodes_per_mode[k] : maxN; }
  for (int k = 1; k < d; ++k) maxS = samples_for(p, k) > maxS ? samples_for(p, k) : maxS;
  int capL[TTQ_MAXD + 1];
  for (int k = 0; k <= d; ++k) capL[k] = (k == 0 || k == d) ? 1 : cap;
  // several pivots per sweep: every interface holds npiv searches' scratch,
  // search j's j strides (the largest of any interface) past search 0's
  const int np = npiv_of(p);
  size_t cs_st = 0, im_st = 0;
  for (int k = 1; k < d; ++k) {
    size_t nc = (size_t)samples_for(p, k);
    const size_t ncol = (size_t)cap * p->nodes_per_mode[k - 1], nrow = (size_t)p->nodes_per_mode[k] * cap;
    nc = nc > ncol ? nc : ncol;
    nc = nc > nrow ? nc : nrow;
    cs_st = nc > cs_st ? nc : cs_st;
    const size_t nchk = (p->nodes_per_mode[k - 1] + 31) / 32, nchk1 = (p->nodes_per_mode[k] + 31) / 32;
    const size_t ni = (size_t)cap * (nchk > nchk1 ? nchk : nchk1);
    im_st = ni > im_st ? ni : im_st;
  }
  L->cs_st = cs_st;
  L->im_st = im_st;
  L->pt_st = maxN;
  Bump b;
  L->dev = b.take(sizeof(Dev));
  L->st = b.take(sizeof(State));
  L->x = b.take(sumN * 8);
  L->w = b.take(sumN * 8);
  L->c = b.take(sumN * 8);
  L->T = b.take((size_t)maxN * 8);
  for (int k = 1; k < d; ++k) {
    L->lidx[k] = b.take((size_t)cap * d * 4);
    L->ridx[k] = b.take((size_t)cap * d * 4);
    L->lpar[k] = b.take((size_t)cap * 4);
    L->lnode[k] = b.take((size_t)cap * 4);
    L->rpar[k] = b.take((size_t)cap * 4);
    L->rnode[k] = b.take((size_t)cap * 4);
  }
  for (int k = 1; k <= d; ++k) {
    L->Y[k] = b.take((size_t)capL[k - 1] * p->nodes_per_mode[k - 1] * capL[k] * 8);
    L->V[k] = b.take((size_t)capL[k - 1] * capL[k] * 8);
    L->Vlo[k] = b.take((size_t)capL[k - 1] * capL[k] * 8);
  }
  {
    size_t tot = 0;
    for (int k = 1; k <= d; ++k) tot += (size_t)capL[k - 1] * capL[k];
    L->vcnt_bytes = tot * 4;
    L->vcnt_all = b.take(L->vcnt_bytes);
    size_t off = 0;
    for (int k = 1; k <= d; ++k) {
      L->vcnt[k] = L->vcnt_all + off * 4;
      off += (size_t)capL[k - 1] * capL[k];
    }
  }
  for (int k = 1; k < d; ++k) {
    L->Qr[k] = b.take((size_t)cap * cap * 8);
    L->Qc[k] = b.take((size_t)cap * cap * 8);
    L->Rc[k] = b.take((size_t)cap * cap * 8);
    L->Rr[k] = b.take((size_t)cap * cap * 8);
    L->Cc[k] = b.take((size_t)cap * cap * 8);
    L->Sr[k] = b.take((size_t)cap * cap * 8);
    L->rinv[k] = b.take((size_t)cap * 8);
    L->zvec[k] = b.take((size_t)cap * np * 8);
    L->pvec[k] = b.take((size_t)cap * 8);
    L->ptab[k] = b.take(((size_t)(np - 1) * maxN +
                         (p->nodes_per_mode[k - 1] > p->nodes_per_mode[k] ? p->nodes_per_mode[k - 1] : p->nodes_per_mode[k])) * 8);
    size_t nc = (size_t)samples_for(p, k);
    size_t ncol = (size_t)cap * p->nodes_per_mode[k - 1], nrow = (size_t)p->nodes_per_mode[k] * cap;
    nc = nc > ncol ? nc : ncol;
    nc = nc > nrow ? nc : nrow;
    L->cs[k] = b.take((nc + (size_t)(np - 1) * cs_st) * 8);
    L->ce[k] = b.take((nc + (size_t)(np - 1) * cs_st) * 8);
    L->zs[k] = b.take((size_t)samples_for(p, k) * cap * 8);
    // per-row maxima of a rook step: one slot per outer index and row of 32 nodes
    const size_t nchk = (p->nodes_per_mode[k - 1] + 31) / 32;
    const size_t nchk1 = (p->nodes_per_mode[k] + 31) / 32;
    L->im[k] = b.take(((size_t)cap * (nchk > nchk1 ? nchk : nchk1) + (size_t)(np - 1) * im_st) * 8);
    const size_t dd = p->precision == TTQ_PREC_DD ? 1 : 0;
    L->luh[k] = b.take(dd * cap * cap * 8);          // double-double LU of G_k (final contraction)
    L->lul[k] = b.take(dd * cap * cap * 8);
    L->lup[k] = b.take(dd * cap * 4);
  }
  const int nch = (maxN + TTQ_CHUNK - 1) / TTQ_CHUNK;
  auto clampi = [](long v, long lo, long hi) { return (int)(v < lo ? lo : (v > hi ? hi : v)); };
  L->sblocks = clampi((maxS + TTQ_WARPS * TTQ_SPW - 1) / (TTQ_WARPS * TTQ_SPW), 1, 64);
  // the rook kernels spread every interface's work over one grid per instance
  L->cblocks = clampi(((long)(d - 1) * cap * nch + TTQ_WARPS - 1) / TTQ_WARPS, 1, 456);
  L->rblocks = L->cblocks;
  L->cbuf = b.take((size_t)4 * cap * 8);
  L->itx = b.take((size_t)(np - 1) * TTQ_MAXD * sizeof(IfaceState));
  L->devs = b.take(sizeof(Dev *));
  L->total = (b.off + 255) & ~(size_t)255;
}

extern "C" int ttq_workspace_bytes(const ttq_problem *p, size_t *bytes) {
  int rc = validate(p);
  if (rc) return rc;
  if (!bytes) return set_err(TTQ_ERR_INVALID_ARG, "null bytes");
  Layout L;
  make_layout(p, &L);
  *bytes = L.total;
  return TTQ_OK;
}

static bool uniform_pair_table(const ttq_problem *p, const double *x) {
  if (p->family != TTQ_FAMILY_D || p->form != TTQ_FORM_RN) return false;
  const int d = p->d, N = p->nodes_per_mode[0];
  for (int k = 1; k < d; ++k) {
    if (p->nodes_per_mode[k] != N) return false;
    for (int i = 0; i < N; ++i)
      if (x[(size_t)k * N + i] != x[i]) return false;
  }
  // every difference x[a] - x[b] must equal +-(x[|a-b|] - x[0]) exactly
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      double dlt = x[a] - x[b];
      double ref = (a >= b) ? (x[a - b] - x[0]) : -(x[b - a] - x[0]);
      if (dlt != ref) return false;
    }
  return true;
}

// ---------------------------------------------------------------------------

static double family_constant(const ttq_problem *p) {
  if (p->family == TTQ_FAMILY_TEST) return 1.0;
  if (p->form == TTQ_FORM_RN) {
    double f = 1.0;
    for (int q = 2; q <= p->n; ++q) f *= q;
    return 4.0 / f;
  }
  return 2.0;
}

// Host descriptor of one instance laid out at `base` (device pointers only; nothing is copied).
static void fill_descriptor(const ttq_problem *p, const double *hx, char *base, const Layout &L,
                            int q_in_smem, Dev &D) {
  const int d = p->d;
  memset(&D, 0, sizeof(D));
  D.d = d; D.family = p->family; D.form = p->form; D.n = p->n; D.cap = p->rank_cap;
  D.rook_max = p->rook_max; D.init_samples = p->init_samples; D.conv_window = p->conv_window;
  D.r0 = p->r0 < 1 ? 1 : p->r0;
  D.wait_ns = 1000000000ULL;                // 1 s: far beyond any search (at most a few ms)
  D.max_sweeps = p->max_sweeps; D.prec = p->precision;
  D.tol = p->tol; D.pivot_tol = p->pivot_tol; D.seed = p->seed;
  D.constant = family_constant(p);
  D.uniformT = uniform_pair_table(p, hx) ? 1 : 0;
  D.sblocks = L.sblocks; D.cblocks = L.cblocks; D.rblocks = L.rblocks;
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      D.sms = sms;
    else
      D.sms = 0;
    cudaGetLastError();
  }
  D.q_in_smem = q_in_smem;
  D.npiv = npiv_of(p);
  D.cs_st = L.cs_st;
  D.im_st = L.im_st;
  D.pt_st = L.pt_st;
  int off = 0;
  for (int k = 0; k < d; ++k) { D.N[k] = p->nodes_per_mode[k]; D.off[k] = off; off += D.N[k]; }
  for (int k = 1; k < d; ++k) D.S[k] = samples_for(p, k);
  for (int k = 0; k <= d; ++k) D.capL[k] = (k == 0 || k == d) ? 1 : p->rank_cap;
  D.x = (const double *)(base + L.x); D.w = (const double *)(base + L.w);
  D.c = (const double *)(base + L.c); D.T = (const double *)(base + L.T);
  for (int k = 1; k < d; ++k) {
    D.lidx[k] = (int *)(base + L.lidx[k]); D.ridx[k] = (int *)(base + L.ridx[k]);
    D.lpar[k] = (int *)(base + L.lpar[k]); D.lnode[k] = (int *)(base + L.lnode[k]);
    D.rpar[k] = (int *)(base + L.rpar[k]); D.rnode[k] = (int *)(base + L.rnode[k]);
    D.Qr[k] = (double *)(base + L.Qr[k]); D.Qc[k] = (double *)(base + L.Qc[k]);
    D.Rc[k] = (double *)(base + L.Rc[k]); D.Rr[k] = (double *)(base + L.Rr[k]);
    D.Cc[k] = (double *)(base + L.Cc[k]); D.Sr[k] = (double *)(base + L.Sr[k]);
    D.rinv[k] = (double *)(base + L.rinv[k]); D.zvec[k] = (double *)(base + L.zvec[k]);
    D.pvec[k] = (double *)(base + L.pvec[k]);
    D.ptab[k] = (double *)(base + L.ptab[k]);
    D.cs[k] = (double *)(base + L.cs[k]); D.ce[k] = (double *)(base + L.ce[k]);
    D.zs[k] = (double *)(base + L.zs[k]);
    D.im[k] = (double *)(base + L.im[k]);
    D.luh[k] = (double *)(base + L.luh[k]); D.lul[k] = (double *)(base + L.lul[k]);
    D.lup[k] = (int *)(base + L.lup[k]);
  }
  for (int k = 1; k <= d; ++k) {
    D.Y[k] = (double *)(base + L.Y[k]); D.V[k] = (double *)(base + L.V[k]); D.Vlo[k] = (double *)(base + L.Vlo[k]);
    D.vcnt[k] = (unsigned *)(base + L.vcnt[k]);
  }
  D.st = (State *)(base + L.st);
  D.cbuf = (double *)(base + L.cbuf);
  D.itx = (IfaceState *)(base + L.itx);
}

// host copies of a problem's nodes and weights (checked finite)
static int host_inputs(const ttq_problem *p, cudaStream_t s, std::vector<double> &hx, std::vector<double> &hw) {
  size_t sumN = 0;
  for (int k = 0; k < p->d; ++k) sumN += p->nodes_per_mode[k];
  hx.resize(sumN);
  hw.resize(sumN);
  if (p->inputs_on_device) {
    CK(cudaMemcpyAsync(hx.data(), p->nodes, sumN * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hw.data(), p->weights, sumN * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  } else {
    memcpy(hx.data(), p->nodes, sumN * 8);
    memcpy(hw.data(), p->weights, sumN * 8);
  }
  for (size_t q = 0; q < sumN; ++q)
    if (!isfinite(hx[q]) || !isfinite(hw[q])) return set_err(TTQ_ERR_INVALID_ARG, "non-finite node or weight");
  return TTQ_OK;
}

// launch configuration from the instances' problems (maxima over the set)
// The dynamic shared memory a kernel may take is a property of the function,
// shared by every plan of the process: it is only ever raised, so a plan made
// later with smaller factors does not lower it under one made earlier.
static std::mutex g_smem_mu;
template <typename K>
static cudaError_t allow_smem(K kern, int bytes) {
  std::lock_guard<std::mutex> lk(g_smem_mu);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  if (bytes <= fa.maxDynamicSharedSizeBytes) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

static void configure(ttq_plan *P, const ttq_problem *probs, int count, const Layout *Ls) {
  P->max_ni = 0; P->rook_max = 1; P->max_sweeps = 1; P->max_cap = 1; P->max_sum_n = 1; P->npiv = 1;
  P->tsm_smem = 0;
  P->rook_rmax = 4;
  P->sblocks = P->cblocks = P->rblocks = 1;
  size_t maxfib = 0;
  for (int q = 0; q < count; ++q) {
    const ttq_problem *p = probs + q;
    const int cap = p->rank_cap;
    P->max_ni = p->d - 1 > P->max_ni ? p->d - 1 : P->max_ni;
    P->rook_max = p->rook_max > P->rook_max ? p->rook_max : P->rook_max;
    P->max_sweeps = p->max_sweeps > P->max_sweeps ? p->max_sweeps : P->max_sweeps;
    P->max_cap = cap > P->max_cap ? cap : P->max_cap;
    P->npiv = npiv_of(p) > P->npiv ? npiv_of(p) : P->npiv;
    int sn = 0;
    for (int k = 0; k < p->d; ++k) sn += p->nodes_per_mode[k];
    P->max_sum_n = sn > P->max_sum_n ? sn : P->max_sum_n;
    if (p->family == TTQ_FAMILY_D && p->form == TTQ_FORM_RN) {
      bool eqN = true;
      for (int k = 1; k < p->d; ++k) eqN = eqN && p->nodes_per_mode[k] == p->nodes_per_mode[0];
      const int tb = eqN ? p->nodes_per_mode[0] * 8 : 0;
      P->tsm_smem = tb > P->tsm_smem ? tb : P->tsm_smem;
    }
    size_t fib = 0;
    for (int k = 1; k <= p->d; ++k) fib += (size_t)((k == 1) ? 1 : cap) * ((k == p->d) ? 1 : cap);
    maxfib = fib > maxfib ? fib : maxfib;
    P->sblocks = Ls[q].sblocks > P->sblocks ? Ls[q].sblocks : P->sblocks;
    P->cblocks = Ls[q].cblocks > P->cblocks ? Ls[q].cblocks : P->cblocks;
  }
  // rook kernels: the device's resident CTA slots (a multiple of the SM count, so
  // the round-robin item deal spreads evenly over the SMs), shared by the instances
  {
    int dev = 0, sms = 152, occ = 3;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rook_col<false>, TTQ_WARPS * 32, 0) != cudaSuccess ||
        occ < 1)
      occ = 1;
    const int slots = sms * occ;
    // one instance: the resident slots less the two of the contraction chains,
    // which may still run on the second stream when the first rook step starts
    if (count == 1) P->cblocks = std::max(sms, slots - 2);
    else P->cblocks = std::min(P->cblocks, std::max(1, (slots + count - 1) / count));
    // evaluation kernel: the same deal, its grid the resident slots when one
    // instance runs less one slot per interface, so that the QR row appends
    // (one CTA per interface, on the second stream) find room beside it at once
    // instead of waiting for its CTAs to retire
    int occe = 3;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occe, k_eval_slabs, TTQ_WARPS * 32, P->tsm_smem) != cudaSuccess ||
        occe < 1)
      occe = 1;
    size_t ge = (maxfib + TTQ_WARPS - 1) / TTQ_WARPS;
    ge = ge < 1 ? 1 : ge;
    P->grid_eval = count == 1 ? std::max(sms, sms * occe - P->max_ni)
                              : (int)std::min(ge, (size_t)std::max(1, (sms * occe + count - 1) / count));
    // samples: at least enough CTAs per interface to fill the resident slots
    // once (each CTA holds one interface's factors), so no SM runs twice the
    // CTAs of another while others idle
    int occs = 1;
    const size_t cap0 = P->max_cap;
    const size_t ssm = (((cap0 <= 96) ? 2 : 1) * cap0 * cap0 + (size_t)TTQ_WARPS * TTQ_SPW * 2 * (cap0 + 1)) * 8;
    allow_smem(k_samples, (int)ssm);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occs, k_samples, TTQ_WARPS * 32, ssm) != cudaSuccess || occs < 1)
      occs = 1;
    const int per = (sms * occs) / std::max(1, P->max_ni * count);
    P->sblocks = std::max(P->sblocks, per);
    cudaGetLastError();
  }
  P->rblocks = P->cblocks;
  const size_t cap = P->max_cap;
  const int q_in = cap <= 96 ? 1 : 0;
  P->qr_smem = (int)((cap * (cap + 1) + 8 * cap) * 8);   // full QR: r(r+1)+r, bordering: r^2+7r
  // R (and Q when it fits), then per warp TTQ_SPW groups of two vectors of cap + 1
  P->samples_smem = (int)(((q_in ? 2 : 1) * cap * cap + (size_t)TTQ_WARPS * TTQ_SPW * 2 * (cap + 1)) * 8);
  P->contract_smem = (int)(cap * cap * 8);
  P->solve_smem = (int)((q_in ? 2 : 1) * cap * cap * 8);
  // persistent search: R D^-1 (and Q) of the group's interface for the whole
  // launch, then the samples' group vectors or the rook scratch in one region
  {
    const size_t vec = (size_t)TTQ_WARPS * TTQ_SPW * 2 * (cap + 1) * 8;
    const size_t scr = vec > sizeof(RookSmem) ? vec : sizeof(RookSmem);
    P->search_smem = (int)((q_in ? 2 : 1) * cap * cap * 8 + scr);
    int dev = 0, sms = 152, occ = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    allow_smem(k_search, P->search_smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_search, TTQ_WARPS * 32, P->search_smem) != cudaSuccess)
      occ = 0;
    // the resident CTA slots less two for the contraction's chains on the second stream
    P->search_grid = occ >= 1 ? sms * occ - 2 : 0;
    P->persistent = 0;                      // opt in with ttq_plan_set_search: measured slower than the staged launches
    cudaGetLastError();
  }
}

static cudaError_t set_smem_attributes(ttq_plan *P) {
  cudaError_t e;
  if ((e = allow_smem(k_qr<false>, P->qr_smem)) != cudaSuccess) return e;
  if ((e = allow_smem(k_qr<true>, P->qr_smem)) != cudaSuccess) return e;
  if ((e = allow_smem(k_qr_row, P->qr_smem)) != cudaSuccess) return e;
  if ((e = allow_smem(k_solve<false>, P->solve_smem)) != cudaSuccess) return e;
  if ((e = allow_smem(k_solve<true>, P->solve_smem)) != cudaSuccess) return e;
  if ((e = allow_smem(k_samples, P->samples_smem)) != cudaSuccess) return e;
  if ((e = allow_smem(k_contract, P->contract_smem)) != cudaSuccess) return e;
  if ((e = allow_smem(k_search, P->search_smem)) != cudaSuccess) return e;
  return allow_smem(k_eval_slabs, P->tsm_smem);   // the pair table's room
}

static void plan_free(ttq_plan *P) {
  if (!P) return;
  if (!P->pending.empty()) cudaStreamSynchronize(P->stream);
  harvest(P);
  for (cudaEvent_t e : P->pool) cudaEventDestroy(e);
  if (P->sweep_exec) cudaGraphExecDestroy(P->sweep_exec);
  if (P->run_exec) cudaGraphExecDestroy(P->run_exec);
  if (P->s2) { cudaStreamSynchronize(P->s2); cudaStreamDestroy(P->s2); }
  if (P->fork) cudaEventDestroy(P->fork);
  if (P->join) cudaEventDestroy(P->join);
  if (P->slots) cudaFreeHost(P->slots);
  if (P->hst) cudaFreeHost(P->hst);
  if (P->count > 1) {
    delete[] P->hs;
    delete[] P->sts;
  }
  delete P;
}

// Instances laid out one after another in `workspace`: an optional array of
// descriptor pointers for the set, then each instance's own layout.
static int plan_build(const ttq_problem *probs, int count, void *workspace, size_t bytes, void *stream,
                      ttq_plan **out) {
  if (count < 1 || count > 65535) return set_err(TTQ_ERR_INVALID_ARG, "count must be in 1..65535");
  if (!out) return set_err(TTQ_ERR_INVALID_ARG, "null out");
  std::vector<Layout> Ls(count);
  size_t need = batch_head_bytes(count);
  std::vector<size_t> offs(count);
  for (int q = 0; q < count; ++q) {
    int rc = validate(probs + q);
    if (rc) return rc;
    if (count > 1 && npiv_of(probs + q) > 1)
      return set_err(TTQ_ERR_INVALID_ARG, "several pivots per sweep: single-instance plans only");
    make_layout(probs + q, &Ls[q]);
    offs[q] = need;
    need += Ls[q].total;
  }
  if (!workspace || bytes < need || ((uintptr_t)workspace & 255))
    return set_err(TTQ_ERR_WORKSPACE, "workspace too small or not 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  ttq_plan *P = new ttq_plan();
  P->count = count;
  P->stream = s;
  configure(P, probs, count, Ls.data());
  P->hs = count == 1 ? &P->h : new Dev[count];
  P->sts = count == 1 ? &P->st : new State *[count];
  char *base0 = (char *)workspace;
  std::vector<Dev *> devp(count);
  cudaError_t e = cudaSuccess;
  int rc = TTQ_OK;
  if (cudaMallocHost((void **)&P->hst, sizeof(State) * count) != cudaSuccess) {
    P->hst = nullptr;
    plan_free(P);
    return set_err(TTQ_ERR_CUDA, "cudaMallocHost failed");
  }
  for (int q = 0; q < count && !rc; ++q) {
    const ttq_problem *p = probs + q;
    char *base = base0 + offs[q];
    std::vector<double> hx, hw;
    if ((rc = host_inputs(p, s, hx, hw))) break;
    fill_descriptor(p, hx.data(), base, Ls[q], P->max_cap <= 96 ? 1 : 0, P->hs[q]);
    devp[q] = (Dev *)(base + Ls[q].dev);
    P->sts[q] = P->hs[q].st;
    const size_t sumN = hx.size();
    if ((e = cudaMemcpyAsync(base + Ls[q].x, hx.data(), sumN * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(base + Ls[q].w, hw.data(), sumN * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(P->hs[q].st, 0, sizeof(State), s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(base + Ls[q].vcnt_all, 0, Ls[q].vcnt_bytes, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(devp[q], &P->hs[q], sizeof(Dev), cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    P->h2d += (long long)(2 * sumN * 8 + sizeof(Dev));
    if (p->inputs_on_device) P->d2h += (long long)(2 * sumN * 8);
    // this instance's own one-entry descriptor array
    Dev **own = (Dev **)(base + Ls[q].devs);
    if ((e = cudaMemcpyAsync(own, &devp[q], sizeof(Dev *), cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if (count == 1) P->devs = own;
    // each host copy's transfers must finish before hx/hw go out of scope
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
  }
  if (!rc && e == cudaSuccess && count > 1) {
    P->devs = (Dev **)base0;
    e = cudaMemcpyAsync(P->devs, devp.data(), count * sizeof(Dev *), cudaMemcpyHostToDevice, s);
    P->h2d += (long long)(count * sizeof(Dev *));
    // the same descriptors in cost order, for the concurrent groups of the run graph
    P->order.resize(count);
    for (int q = 0; q < count; ++q) P->order[q] = q;
    std::stable_sort(P->order.begin(), P->order.end(),
                     [&](int a, int b) { return instance_cost(probs + a) < instance_cost(probs + b); });
    std::vector<Dev *> sorted(count);
    for (int q = 0; q < count; ++q) sorted[q] = devp[P->order[q]];
    P->devs_sorted = (Dev **)(base0 + batch_head_bytes(count) / 2);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(P->devs_sorted, sorted.data(), count * sizeof(Dev *), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    P->h2d += (long long)(count * sizeof(Dev *));
    P->ngroups = std::min(8, count / 32 > 1 ? count / 32 : 1);
  }
  if (!rc && e == cudaSuccess) {
    P->h = P->hs[0];
    P->dev = devp[0];
    P->st = P->sts[0];
    P->guard = (unsigned *)((char *)P->sts[0] + offsetof(State, batch_guard));
    if ((e = set_smem_attributes(P)) == cudaSuccess &&
        (e = create_side_stream(&P->s2, count == 1)) == cudaSuccess &&
        (e = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming)) == cudaSuccess &&
        (e = cudaEventCreateWithFlags(&P->join, cudaEventDisableTiming)) == cudaSuccess) {
      P->use_graph = s != nullptr ? 1 : 0;   // no capture on the legacy default stream
      timed(P, KT_SETUP, [&] {
        k_setup<<<dim3((P->max_sum_n + 255) / 256, 1, count), 256, 0, s>>>(P->devs);
      });
      if ((e = cudaGetLastError()) == cudaSuccess) e = cudaStreamSynchronize(s);
    }
  }
  if (rc || e != cudaSuccess) {
    if (!rc) {
      g_last_error = std::string("plan setup: ") + cudaGetErrorString(e);
      rc = TTQ_ERR_CUDA;
    }
    plan_free(P);
    return rc;
  }
  *out = P;
  return TTQ_OK;
}

extern "C" int ttq_plan_create(const ttq_problem *p, void *workspace, size_t bytes, void *stream, ttq_plan **out) {
  return plan_build(p, 1, workspace, bytes, stream, out);
}

extern "C" int ttq_plan_destroy(ttq_plan *P) {
  plan_free(P);
  return TTQ_OK;
}

extern "C" int ttq_batch_workspace_bytes(const ttq_problem *probs, int count, size_t *bytes) {
  if (!probs || !bytes || count < 1 || count > 65535) return set_err(TTQ_ERR_INVALID_ARG, "bad argument");
  size_t need = batch_head_bytes(count);
  for (int q = 0; q < count; ++q) {
    int rc = validate(probs + q);
    if (rc) return rc;
    Layout L;
    make_layout(probs + q, &L);
    need += L.total;
  }
  *bytes = need;
  return TTQ_OK;
}

extern "C" int ttq_batch_create(const ttq_problem *probs, int count, void *workspace, size_t bytes, void *stream,
                                ttq_plan **out) {
  if (!probs) return set_err(TTQ_ERR_INVALID_ARG, "null problems");
  return plan_build(probs, count, workspace, bytes, stream, out);
}

// ---------------------------------------------------------------------------
// One sequential sweep (Alg. 5), plain launches on the plan's stream: the
// sweep's cores, factors and integral, then per interface k = 1..d-1 the
// staged search with only k searching, its pivot appended at once, and the new
// core slabs and QR update that the append calls for.
static void enqueue_sweep_seq(ttq_plan *P) {
  cudaStream_t s = P->stream;
  const int ni = P->max_ni, nb = P->count;
  Dev *const *dv = P->devs;
  const dim3 W(TTQ_WARPS * 32), T(256);
  auto refresh = [&] {
    timed(P, KT_QR, [&] { k_qr_row<<<dim3(ni, 1, nb), 256, P->qr_smem, s>>>(dv); });
    timed(P, KT_EVAL, [&] { k_eval_slabs<<<dim3(P->grid_eval, 1, nb), W, P->tsm_smem, s>>>(dv); });
    timed(P, KT_QR, [&] { k_qr<false><<<dim3(ni, 1, nb), T, P->qr_smem, s>>>(dv); });
  };
  refresh();
  timed(P, KT_CONTRACT, [&] { k_contract<<<dim3(2, 1, nb), 256, P->contract_smem, s>>>(dv, 0); });
  for (int k = 1; k <= ni; ++k) {
    k_seq_begin<<<dim3(1, 1, nb), 32, 0, s>>>(dv, k);
    P->launches++;
    timed(P, KT_SAMPLES, [&] { k_samples<<<dim3(P->sblocks, ni, nb), W, P->samples_smem, s>>>(dv); });
    for (int q = 0; q < P->rook_max; ++q) {
      timed(P, KT_ROOK_COL, [&] {
        k_rook_col<false><<<dim3(P->cblocks, 1, nb), W, 0, s>>>(dv, P->rook_rmax);
      });
      timed(P, KT_SOLVE, [&] { k_solve<false><<<dim3(ni, 1, nb), T, P->solve_smem, s>>>(dv, 1, 0, P->cond, 0); });
      timed(P, KT_ROOK_ROW, [&] {
        k_rook_row<false><<<dim3(P->rblocks, 1, nb), W, 0, s>>>(dv, P->rook_rmax);
      });
      timed(P, KT_SOLVE, [&] { k_solve<false><<<dim3(ni, 1, nb), T, P->solve_smem, s>>>(dv, 2, 0, P->cond, 0); });
    }
    timed(P, KT_UPDATE, [&] { k_seq_end<<<dim3(1, 1, nb), T, 0, s>>>(dv, k, k == ni ? 1 : 0); });
    if (k < ni) refresh();
  }
}

// ---------------------------------------------------------------------------
// One sweep for every instance: eval -> qr -> { contract (side stream) |
// samples -> rook rounds } -> update.  Every launch covers all instances
// (grid z); CTAs of instances or interfaces with no work exit at once.
static void enqueue_sweep(ttq_plan *P, bool loop_end = true, bool head = false) {
  if (P->sequential) {
    enqueue_sweep_seq(P);
    return;
  }
  cudaStream_t s = P->stream;
  const int ni = P->max_ni, nb = P->cur_dv ? P->cur_nb : P->count;
  Dev *const *dv = P->cur_dv ? P->cur_dv : P->devs;
  const dim3 W(TTQ_WARPS * 32), T(256);
  // the QR row append (old entries only) beside the evaluation of the new slabs
  if (P->s2) {
    cudaEventRecord(P->fork, s);
    cudaStreamWaitEvent(P->s2, P->fork, 0);
    timed_on(P, P->s2, KT_QR, [&] { k_qr_row<<<dim3(ni, 1, nb), 256, P->qr_smem, P->s2>>>(dv); });
    cudaEventRecord(P->join, P->s2);
  } else {
    timed(P, KT_QR, [&] { k_qr_row<<<dim3(ni, 1, nb), 256, P->qr_smem, s>>>(dv); });
  }
  // kernel (a) overlaps its predecessor's tail (programmatic serialization)
  // except as the first node of the run graph's body, where nothing precedes it
  // and a plain launch lets the QR row kernel beside it start at once
  if (P->in_loop && head)
    timed(P, KT_EVAL, [&] { k_eval_slabs<<<dim3(P->grid_eval, 1, nb), W, P->tsm_smem, s>>>(dv); });
  else
    timed(P, KT_EVAL, [&] { launch_k(P, k_eval_slabs, dim3(P->grid_eval, 1, nb), W, P->tsm_smem, s, dv); });
  if (P->s2) cudaStreamWaitEvent(s, P->join, 0);
  const bool multi = P->npiv > 1;
  timed(P, KT_QR, [&] { launch_k(P, multi ? k_qr<true> : k_qr<false>, dim3(ni, 1, nb), T, P->qr_smem, s, dv); });
  if (P->s2) {
    cudaEventRecord(P->fork, s);
    cudaStreamWaitEvent(P->s2, P->fork, 0);
    timed_on(P, P->s2, KT_CONTRACT, [&] { k_contract<<<dim3(2, 1, nb), 256, P->contract_smem, P->s2>>>(dv, 0); });
    cudaEventRecord(P->join, P->s2);
  } else {
    timed(P, KT_CONTRACT, [&] { k_contract<<<dim3(2, 1, nb), 256, P->contract_smem, s>>>(dv, 0); });
  }
  const int single_cond = P->in_loop && loop_end && nb == 1;
  if (P->persistent && nb == 1) {
    // the whole search in one cooperative launch; its end (ranks, stopping
    // rules, the WHILE condition) after the contraction has joined
    timed(P, KT_SEARCH, [&] { launch_k(P, k_search, dim3(P->search_grid, 1, 1), W, (size_t)P->search_smem, s, dv); });
    if (P->s2) cudaStreamWaitEvent(s, P->join, 0);
    timed(P, KT_UPDATE, [&] { k_sweep_end<<<1, T, 0, s>>>(dv, P->cond, single_cond); });
    return;
  }
  // the samples stage ends, per interface, in its last CTA (the best sample and
  // the first column solve); each rook step is followed by the decisions kernel
  timed(P, KT_SAMPLES, [&] { launch_k(P, k_samples, dim3(P->sblocks, ni, nb), W, P->samples_smem, s, dv); });
  // the last decisions kernel also ends the sweep (appends, ranks, stopping
  // rules, the WHILE condition), after the contraction has joined
  for (int q = 0; q < P->rook_max; ++q) {
    const bool fin = q == P->rook_max - 1;
    timed(P, KT_ROOK_COL, [&] {
      launch_k(P, multi ? k_rook_col<true> : k_rook_col<false>, dim3(P->cblocks, 1, nb), W, 0, s, dv, P->rook_rmax);
    });
    timed(P, KT_SOLVE, [&] {
      launch_k(P, multi ? k_solve<true> : k_solve<false>, dim3(ni, P->npiv, nb), T, P->solve_smem, s, dv, 1, 0,
               P->cond, 0);
    });
    timed(P, KT_ROOK_ROW, [&] {
      launch_k(P, multi ? k_rook_row<true> : k_rook_row<false>, dim3(P->rblocks, 1, nb), W, 0, s, dv, P->rook_rmax);
    });
    if (fin && P->s2) cudaStreamWaitEvent(s, P->join, 0);
    timed(P, fin ? KT_UPDATE : KT_SOLVE, [&] {
      launch_k(P, multi ? k_solve<true> : k_solve<false>, dim3(ni, P->npiv, nb), T, P->solve_smem, s, dv, 2,
               fin ? 1 : 0, P->cond,
               fin ? single_cond : 0);
    });
  }
  if (P->in_loop && loop_end && nb > 1) {
    launch_k(P, k_batch_cond, dim3(1), T, 0, s, dv, nb, P->max_sweeps, P->cur_dv ? P->cur_guard : P->guard, P->cond);
    P->launches++;
  }
}

// Whole run as one graph: a conditional WHILE node whose body is four sweeps;
// the condition is set on the device (the last decisions kernel of the sweep for one instance, k_batch_cond
// for a batch), so a run needs no host round trip per sweep.
static int build_run_graph(ttq_plan *P) {
  // a batch split into groups: one WHILE node per group, with no edges between
  // them, so the groups' sweeps run concurrently; each group's condition
  // kernel watches its own instances and counts its iterations in the
  // batch_guard of its first instance's state
  const int G = (P->count > 1 && P->devs_sorted && P->ngroups > 1) ? P->ngroups : 1;
  P->glo.assign(G, 0);
  P->gcnt.assign(G, P->count);
  P->gkernels.assign(G, 0);
  if (G > 1)
    for (int g = 0; g < G; ++g) {
      P->glo[g] = (int)((long long)g * P->count / G);
      P->gcnt[g] = (int)((long long)(g + 1) * P->count / G) - P->glo[g];
    }
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  const long long l0 = P->launches;
  long long n0[KT_N];
  memcpy(n0, P->kt_n, sizeof(n0));
  cudaError_t e = cudaSuccess;
  for (int grp = 0; grp < G && e == cudaSuccess; ++grp) {
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { g_last_error = std::string("conditional handle: ") + cudaGetErrorString(e); break; }
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    memset(npbuf, 0, sizeof(npbuf));
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(npbuf);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) { g_last_error = std::string("while node: ") + cudaGetErrorString(e); break; }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    P->cond = h;
    P->in_loop = 1;
    if (G > 1) {
      P->cur_dv = P->devs_sorted + P->glo[grp];
      P->cur_nb = P->gcnt[grp];
      P->cur_guard = (unsigned *)((char *)P->sts[P->order[P->glo[grp]]] + offsetof(State, batch_guard));
    }
    const long long lg = P->launches;
    // four sweeps per iteration: the condition is evaluated (and the body
    // relaunched, ~5 us) a quarter as often; a sweep that follows the stop
    // finds it set and its kernels return at once
    e = cudaStreamBeginCaptureToGraph(P->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      enqueue_sweep(P, false, true);
      enqueue_sweep(P, false);
      enqueue_sweep(P, false);
      enqueue_sweep(P, true);
      e = cudaStreamEndCapture(P->stream, &body);
    }
    P->gkernels[grp] = (int)(P->launches - lg);
    P->in_loop = 0;
    P->cur_dv = nullptr;
    if (e != cudaSuccess) g_last_error = std::string("run graph: ") + cudaGetErrorString(e);
  }
  P->sweep_kernels = (int)(P->launches - l0);
  P->launches = l0;
  memcpy(P->kt_n, n0, sizeof(n0));
  if (e == cudaSuccess) {
    e = cudaGraphInstantiate(&P->run_exec, g, cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) g_last_error = std::string("run graph: ") + cudaGetErrorString(e);
  }
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return TTQ_ERR_CUDA;
  return TTQ_OK;
}

static int launch_sweep(ttq_plan *P) {
  if (P->use_graph && !P->timing && P->count == 1 && !P->sequential) {
    if (!P->sweep_exec) {
      cudaGraph_t g = nullptr;
      const long long l0 = P->launches;
      long long n0[KT_N];
      memcpy(n0, P->kt_n, sizeof(n0));
      CK(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
      enqueue_sweep(P);
      cudaError_t e = cudaStreamEndCapture(P->stream, &g);
      if (e != cudaSuccess) { g_last_error = std::string("sweep capture: ") + cudaGetErrorString(e); return TTQ_ERR_CUDA; }
      const int nk = (int)(P->launches - l0);
      P->launches = l0;
      memcpy(P->kt_n, n0, sizeof(n0));
      e = cudaGraphInstantiate(&P->sweep_exec, g, cudaGraphInstantiateFlagUseNodePriority);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { g_last_error = std::string("sweep graph: ") + cudaGetErrorString(e); return TTQ_ERR_CUDA; }
      P->sweep_kernels = nk;
    }
    CK(cudaGraphLaunch(P->sweep_exec, P->stream));
    P->launches += P->sweep_kernels;
    return TTQ_OK;
  }
  enqueue_sweep(P);
  CK(cudaGetLastError());
  return TTQ_OK;
}

// copy every instance's state to the host mirror and wait
static int read_states(ttq_plan *P) {
  for (int q = 0; q < P->count; ++q)
    CK(cudaMemcpyAsync(P->hst + q, P->sts[q], sizeof(State), cudaMemcpyDeviceToHost, P->stream));
  P->d2h += (long long)sizeof(State) * P->count;
  CK(cudaStreamSynchronize(P->stream));
  harvest(P);
  return TTQ_OK;
}
static int read_state(ttq_plan *P) { return read_states(P); }

extern "C" int ttq_plan_init(ttq_plan *P) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  timed(P, KT_INIT, [&] { k_init<<<dim3(1, 1, P->count), TTQ_WARPS * 32, 0, P->stream>>>(P->devs); });
  CK(cudaGetLastError());
  return TTQ_OK;
}

static void fill_result_from(const Dev &D, const State &S, ttq_result *out) {
  out->value = S.value;
  out->value_lo = S.value_lo;
  out->internal_conv = S.conv;
  long long core = 0;
  int mr = 0;
  for (int k = 1; k <= D.d; ++k) core += (long long)S.r[k - 1] * D.N[k - 1] * S.r[k];
  for (int k = 0; k <= D.d; ++k) mr = S.r[k] > mr ? S.r[k] : mr;
  out->n_eval = core + S.search_evals + S.init_evals;
  out->sweeps = S.nchanges + 1;
  out->max_rank = mr;
  out->status = S.status;
  out->d = D.d;
  for (int k = 0; k <= TTQ_MAX_MODES; ++k) out->ranks[k] = k <= D.d ? S.r[k] : 0;
}

static int any_prec(const ttq_plan *P) {
  for (int q = 0; q < P->count; ++q)
    if (P->hs[q].prec) return 1;
  return 0;
}

// enqueue a whole run of every instance (graph path); returns without waiting
static int enqueue_run(ttq_plan *P) {
  int rc;
  if ((rc = ttq_plan_init(P))) return rc;
  k_begin<<<dim3(1, 1, P->count), 1, 0, P->stream>>>(P->devs, 0, 1, 1);
  P->launches++;
  CK(cudaGetLastError());
  if (!P->run_exec && (rc = build_run_graph(P))) return rc;
  if (P->count > 1 && P->glo.size() > 1) {
    for (size_t g = 0; g < P->glo.size(); ++g)
      CK(cudaMemsetAsync((char *)P->sts[P->order[P->glo[g]]] + offsetof(State, batch_guard), 0, sizeof(unsigned),
                         P->stream));
  } else if (P->count > 1) {
    CK(cudaMemsetAsync(P->guard, 0, sizeof(unsigned), P->stream));
  }
  CK(cudaGraphLaunch(P->run_exec, P->stream));
  if (any_prec(P)) {                        // double-double contraction of the final sets
    timed(P, KT_CONTRACT, [&] { k_dd_factor<<<dim3(P->max_ni, 1, P->count), 256, 0, P->stream>>>(P->devs); });
    timed(P, KT_CONTRACT, [&] { k_contract<<<dim3(2, 1, P->count), 256, P->contract_smem, P->stream>>>(P->devs, 1); });
    CK(cudaGetLastError());
  }
  return TTQ_OK;
}

// run every instance to its stop (blocking); states land in P->hst
static int run_all(ttq_plan *P) {
  int rc;
  if (P->use_graph && !P->timing && !P->sequential) {
    if ((rc = enqueue_run(P))) return rc;
    if ((rc = read_states(P))) return rc;
    if (P->count > 1) {
      // each WHILE loop of the batch: its iterations (its condition kernel's
      // count) times the kernels of one iteration
      const bool grouped = P->glo.size() > 1;
      for (size_t g = 0; g < P->gkernels.size(); ++g) {
        const State &S0 = P->hst[grouped ? P->order[P->glo[g]] : 0];
        P->launches += (long long)P->gkernels[g] * S0.batch_guard;
      }
      return TTQ_OK;
    }
    int mx = 0;
    for (int q = 0; q < P->count; ++q) mx = P->hst[q].loop_guard > mx ? P->hst[q].loop_guard : mx;
    P->launches += (long long)P->sweep_kernels * mx;
    return TTQ_OK;
  }
  if ((rc = ttq_plan_init(P))) return rc;
  k_begin<<<dim3(1, 1, P->count), 1, 0, P->stream>>>(P->devs, 0, 1, 1);
  P->launches++;
  CK(cudaGetLastError());
  const int batch = 2;
  for (int s = 0; s < P->max_sweeps; s += batch) {
    for (int b = 0; b < batch; ++b)
      if ((rc = launch_sweep(P))) return rc;
    int all = 1;
    for (int q = 0; q < P->count; ++q)
      CK(cudaMemcpyAsync(&P->hst[q].stop, &P->sts[q]->stop, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    P->d2h += (long long)sizeof(int) * P->count;
    CK(cudaStreamSynchronize(P->stream));
    harvest(P);
    for (int q = 0; q < P->count; ++q) all &= P->hst[q].stop ? 1 : 0;
    if (all) break;
  }
  if (any_prec(P)) {
    timed(P, KT_CONTRACT, [&] { k_dd_factor<<<dim3(P->max_ni, 1, P->count), 256, 0, P->stream>>>(P->devs); });
    timed(P, KT_CONTRACT, [&] { k_contract<<<dim3(2, 1, P->count), 256, P->contract_smem, P->stream>>>(P->devs, 1); });
    CK(cudaGetLastError());
  }
  return read_states(P);
}

extern "C" int ttq_plan_run(ttq_plan *P, ttq_result *out) {
  if (!P || !out) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  int rc = run_all(P);
  if (rc) return rc;
  fill_result_from(P->hs[0], P->hst[0], out);
  return TTQ_OK;
}

extern "C" int ttq_batch_run(ttq_plan *P, ttq_result *results) {
  if (!P || !results) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  int rc = run_all(P);
  if (rc) return rc;
  for (int q = 0; q < P->count; ++q) fill_result_from(P->hs[q], P->hst[q], results + q);
  return TTQ_OK;
}

extern "C" int ttq_plan_launch(ttq_plan *P, int slot) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  if (P->count != 1) return set_err(TTQ_ERR_INVALID_ARG, "ttq_plan_launch needs a single-instance plan");
  if (slot < 0 || slot >= TTQ_RESULT_SLOTS) return set_err(TTQ_ERR_INVALID_ARG, "slot out of range");
  if (!P->slots) {                          // first launch: pinned result slots (warm up before timing)
    if (cudaMallocHost((void **)&P->slots, sizeof(State) * TTQ_RESULT_SLOTS) != cudaSuccess)
      return set_err(TTQ_ERR_CUDA, "cudaMallocHost failed");
  }
  int rc;
  if (!(P->use_graph && !P->timing && !P->sequential)) {   // plain launches need the host in the loop: run now
    if ((rc = run_all(P))) return rc;
    memcpy(&P->slots[slot], P->hst, sizeof(State));
    return TTQ_OK;
  }
  if ((rc = enqueue_run(P))) return rc;
  CK(cudaMemcpyAsync(&P->slots[slot], P->st, sizeof(State), cudaMemcpyDeviceToHost, P->stream));
  P->d2h += sizeof(State);
  return TTQ_OK;
}

extern "C" int ttq_plan_result(ttq_plan *P, int slot, ttq_result *out) {
  if (!P || !out) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  if (slot < 0 || slot >= TTQ_RESULT_SLOTS || !P->slots) return set_err(TTQ_ERR_INVALID_ARG, "bad slot");
  CK(cudaStreamSynchronize(P->stream));
  harvest(P);
  const State &S = P->slots[slot];
  P->launches += (long long)P->sweep_kernels * S.loop_guard;
  fill_result_from(P->h, S, out);
  return TTQ_OK;
}

// Autotuner: CTAs per interface of the sample and rook kernels and CTAs per
// instance of the evaluation kernel.  Every candidate computes the same
// results (the reductions do not depend on the grid); each is timed with CUDA
// events over `sweeps` sweeps from the initial sets and the fastest kept.
extern "C" int ttq_batch_autotune(ttq_plan *P, int sweeps, int32_t *chosen) {
  if (!P || sweeps < 1) return set_err(TTQ_ERR_INVALID_ARG, "bad argument");
  const int cand_c[] = {4, 16, 38, 76, 152, 304, 456};
  const int cand_s[] = {8, 16, 32, 64, 128};
  const int cand_e[] = {152, 304, 608, 1216};
  const int cand_r[] = {1, 2, 4};
  const int save_timing = P->timing;
  P->timing = 1;
  auto time_cfg = [&](double *ms_out) -> int {
    int rc;
    if ((rc = ttq_plan_init(P))) return rc;
    k_begin<<<dim3(1, 1, P->count), 1, 0, P->stream>>>(P->devs, 0, 1, 1);
    CK(cudaGetLastError());
    double before[KT_N];
    if ((rc = read_states(P))) return rc;
    memcpy(before, P->kt_ms, sizeof(before));
    for (int s = 0; s < sweeps; ++s)
      if ((rc = launch_sweep(P))) return rc;
    if ((rc = read_states(P))) return rc;
    *ms_out = (P->kt_ms[KT_EVAL] - before[KT_EVAL]) + (P->kt_ms[KT_SAMPLES] - before[KT_SAMPLES]) +
              (P->kt_ms[KT_ROOK_COL] - before[KT_ROOK_COL]) + (P->kt_ms[KT_ROOK_ROW] - before[KT_ROOK_ROW]);
    return TTQ_OK;
  };
  // Each dimension in turn: the largest candidate whose time is within 3% of
  // the fastest.  The trial sweeps are the first of the run (low ranks, where
  // the grid size hardly matters and timing noise would decide), while the
  // later, higher-rank sweeps that dominate a run gain from the larger grids.
  int rc = TTQ_OK;
  auto pick = [&](const int *cand, int n, int *target, int *target2) -> int {
    double t[8];
    double best = 1e300;
    for (int q = 0; q < n; ++q) {
      *target = cand[q];
      if (target2) *target2 = cand[q];
      if ((rc = time_cfg(&t[q]))) return cand[0];
      best = t[q] < best ? t[q] : best;
    }
    int chosen = cand[0];
    for (int q = 0; q < n; ++q)
      if (t[q] <= 1.03 * best && cand[q] > chosen) chosen = cand[q];
    return chosen;
  };
  const int bc = pick(cand_c, 7, &P->cblocks, &P->rblocks);
  P->cblocks = P->rblocks = bc;
  int bs = P->sblocks, be = P->grid_eval;
  if (!rc) bs = pick(cand_s, 5, &P->sblocks, nullptr);
  P->sblocks = bs;
  if (!rc) be = pick(cand_e, 4, &P->grid_eval, nullptr);
  P->grid_eval = be;
  int br = P->rook_rmax;
  if (!rc) br = pick(cand_r, 3, &P->rook_rmax, nullptr);
  P->rook_rmax = br;
  P->timing = save_timing;
  for (int k = 0; k < KT_N; ++k) { P->kt_ms[k] = 0.0; P->kt_n[k] = 0; }
  if (P->run_exec) { cudaGraphExecDestroy(P->run_exec); P->run_exec = nullptr; }
  if (P->sweep_exec) { cudaGraphExecDestroy(P->sweep_exec); P->sweep_exec = nullptr; }
  if (chosen) { chosen[0] = P->cblocks; chosen[1] = P->sblocks; chosen[2] = P->grid_eval; chosen[3] = P->rook_rmax; }
  return rc;
}

extern "C" int ttq_batch_set_groups(ttq_plan *P, int groups) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  if (P->count < 2 || !P->devs_sorted) return set_err(TTQ_ERR_INVALID_ARG, "groups need a batch of two or more instances");
  if (groups < 1 || groups > TTQ_MAX_BATCH_GROUPS || groups > P->count / 2 + (groups == 1 ? 1 : 0))
    return set_err(TTQ_ERR_INVALID_ARG, "groups must be in 1..min(8, count / 2)");
  P->ngroups = groups;
  if (P->run_exec) { cudaGraphExecDestroy(P->run_exec); P->run_exec = nullptr; }
  return TTQ_OK;
}

extern "C" int ttq_plan_set_rook_rows(ttq_plan *P, int rmax) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  if (rmax != 1 && rmax != 2 && rmax != 4) return set_err(TTQ_ERR_INVALID_ARG, "rook item rows must be 1, 2 or 4");
  P->rook_rmax = rmax;
  if (P->run_exec) { cudaGraphExecDestroy(P->run_exec); P->run_exec = nullptr; }
  if (P->sweep_exec) { cudaGraphExecDestroy(P->sweep_exec); P->sweep_exec = nullptr; }
  return TTQ_OK;
}

extern "C" int ttq_plan_set_config(ttq_plan *P, int rook_ctas, int sample_ctas, int eval_ctas) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  if (rook_ctas < 1 || rook_ctas > 65535 || sample_ctas < 1 || sample_ctas > 65535 || eval_ctas < 1 ||
      eval_ctas > 65535)
    return set_err(TTQ_ERR_INVALID_ARG, "CTA counts out of range");
  P->cblocks = P->rblocks = rook_ctas;
  P->sblocks = sample_ctas;
  P->grid_eval = eval_ctas;
  if (P->run_exec) { cudaGraphExecDestroy(P->run_exec); P->run_exec = nullptr; }
  if (P->sweep_exec) { cudaGraphExecDestroy(P->sweep_exec); P->sweep_exec = nullptr; }
  return TTQ_OK;
}

extern "C" int ttq_plan_sweep(ttq_plan *P, int sweep_index, int search, double *value, double *value_lo,
                              ttq_pivot *pivots) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  if (P->count != 1) return set_err(TTQ_ERR_INVALID_ARG, "stage calls need a single-instance plan");
  k_begin<<<1, 1, 0, P->stream>>>(P->devs, sweep_index, 0, search ? 1 : 0);
  P->launches++;
  int rc = launch_sweep(P);
  if (rc) return rc;
  if (P->h.prec && !search) {               // this sweep's sets, contracted in double-double
    if (P->s2) CK(cudaStreamSynchronize(P->s2));
    timed(P, KT_CONTRACT, [&] { k_dd_factor<<<P->max_ni, 256, 0, P->stream>>>(P->devs); });
    timed(P, KT_CONTRACT, [&] { k_contract<<<2, 256, P->contract_smem, P->stream>>>(P->devs, 1); });
    CK(cudaGetLastError());
  }
  if ((rc = read_state(P))) return rc;
  const State &S = *P->hst;
  if (value) *value = S.value;
  if (value_lo) *value_lo = S.value_lo;
  if (pivots) {
    for (int k = 1; k < P->h.d; ++k) {
      const IfaceState &I = S.it[k];
      ttq_pivot &pv = pivots[k - 1];
      pv.k = k;
      pv.searched = I.active;
      pv.row = I.row;
      pv.col = I.col;
      pv.err = I.err;
      pv.accepted = I.accepted;
      pv.rounds = I.rounds;
      pv.evals = (int64_t)I.evals;
    }
  }
  if (S.status < 0)
    return set_err(S.status, S.status == ST_ERR_SINGULAR ? "singular cross matrix"
                             : S.status == ST_ERR_TIMEOUT ? "a wait between CTAs passed its limit"
                                                          : "non-finite integrand");
  return TTQ_OK;
}

extern "C" int ttq_plan_set_state(ttq_plan *P, const int32_t *ranks, const int32_t *lpar, const int32_t *lnode,
                                  const int32_t *rpar, const int32_t *rnode) {
  if (P && P->count != 1) return set_err(TTQ_ERR_INVALID_ARG, "stage calls need a single-instance plan");
  if (!P || !ranks || !lpar || !lnode || !rpar || !rnode) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  const Dev &D = P->h;
  const int d = D.d;
  if (ranks[0] != 1 || ranks[d] != 1) return set_err(TTQ_ERR_INVALID_ARG, "ranks[0] and ranks[d] must be 1");
  std::vector<std::vector<int>> L(d + 1), R(d + 2);
  L[0] = std::vector<int>();
  size_t o = 0;
  std::vector<size_t> offs(d + 1, 0);
  for (int k = 1; k < d; ++k) {
    if (ranks[k] < 1 || ranks[k] > D.cap) return set_err(TTQ_ERR_INVALID_ARG, "rank out of range");
    offs[k] = o;
    o += ranks[k];
  }
  // rebuild the full multi-index rows and validate nestedness
  std::vector<std::vector<int>> lrows(d + 1), rrows(d + 2);
  lrows[0] = std::vector<int>(d, -1);
  for (int k = 1; k < d; ++k) {
    lrows[k].assign((size_t)ranks[k] * d, -1);
    for (int a = 0; a < ranks[k]; ++a) {
      int par = lpar[offs[k] + a], nd = lnode[offs[k] + a];
      if (par < 0 || par >= ranks[k - 1] || nd < 0 || nd >= D.N[k - 1]) return set_err(TTQ_ERR_INVALID_ARG, "bad left parent");
      for (int m = 0; m < k - 1; ++m) lrows[k][(size_t)a * d + m] = lrows[k - 1][(size_t)par * d + m];
      lrows[k][(size_t)a * d + k - 1] = nd;
    }
  }
  rrows[d] = std::vector<int>(d, -1);
  for (int k = d - 1; k >= 1; --k) {
    rrows[k].assign((size_t)ranks[k] * d, -1);
    for (int b = 0; b < ranks[k]; ++b) {
      int par = rpar[offs[k] + b], nd = rnode[offs[k] + b];
      if (par < 0 || par >= ranks[k + 1] || nd < 0 || nd >= D.N[k]) return set_err(TTQ_ERR_INVALID_ARG, "bad right parent");
      rrows[k][(size_t)b * d + k] = nd;
      for (int m = k + 1; m < d; ++m) rrows[k][(size_t)b * d + m] = rrows[k + 1][(size_t)par * d + m];
    }
  }
  cudaStream_t s = P->stream;
  for (int k = 1; k < d; ++k) {
    CK(cudaMemcpyAsync(D.lidx[k], lrows[k].data(), lrows[k].size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.ridx[k], rrows[k].data(), rrows[k].size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.lpar[k], lpar + offs[k], ranks[k] * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.lnode[k], lnode + offs[k], ranks[k] * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.rpar[k], rpar + offs[k], ranks[k] * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.rnode[k], rnode + offs[k], ranks[k] * 4, cudaMemcpyHostToDevice, s));
  }
  State *h = P->hst;
  memset(h, 0, sizeof(State));
  for (int k = 0; k <= d; ++k) { h->r[k] = ranks[k]; h->ro[k] = 0; }
  h->conv = INFINITY;
  CK(cudaMemcpyAsync(P->st, h, sizeof(State), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return TTQ_OK;
}

extern "C" int ttq_plan_get_state(ttq_plan *P, int32_t *ranks, int32_t *lpar, int32_t *lnode, int32_t *rpar,
                                  int32_t *rnode) {
  if (P && P->count != 1) return set_err(TTQ_ERR_INVALID_ARG, "stage calls need a single-instance plan");
  if (!P || !ranks) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  int rc = read_state(P);
  if (rc) return rc;
  const Dev &D = P->h;
  const int d = D.d;
  for (int k = 0; k <= d; ++k) ranks[k] = P->hst->r[k];
  size_t o = 0;
  for (int k = 1; k < d; ++k) {
    int r = ranks[k];
    if (lpar) CK(cudaMemcpy(lpar + o, D.lpar[k], r * 4, cudaMemcpyDeviceToHost));
    if (lnode) CK(cudaMemcpy(lnode + o, D.lnode[k], r * 4, cudaMemcpyDeviceToHost));
    if (rpar) CK(cudaMemcpy(rpar + o, D.rpar[k], r * 4, cudaMemcpyDeviceToHost));
    if (rnode) CK(cudaMemcpy(rnode + o, D.rnode[k], r * 4, cudaMemcpyDeviceToHost));
    o += r;
  }
  return TTQ_OK;
}

extern "C" int ttq_plan_get_core(ttq_plan *P, int k, double *host_out) {
  if (P && P->count != 1) return set_err(TTQ_ERR_INVALID_ARG, "stage calls need a single-instance plan");
  if (!P || !host_out) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  const Dev &D = P->h;
  if (k < 1 || k > D.d) return set_err(TTQ_ERR_INVALID_ARG, "k out of range");
  int rc = read_state(P);
  if (rc) return rc;
  const int rl = P->hst->ro[k - 1], rr = P->hst->ro[k], Nk = D.N[k - 1];
  std::vector<double> buf((size_t)D.capL[k - 1] * Nk * D.capL[k]);
  CK(cudaMemcpy(buf.data(), D.Y[k], buf.size() * 8, cudaMemcpyDeviceToHost));
  for (int a = 0; a < rl; ++a)
    for (int i = 0; i < Nk; ++i)
      for (int b = 0; b < rr; ++b)
        host_out[((size_t)a * Nk + i) * rr + b] = buf[((size_t)b * D.capL[k - 1] + a) * Nk + i];
  return TTQ_OK;
}

// ---------------------------------------------------------------------------
// The tensor train as a result (Alg. 6's output: cores and nested index sets)

struct ttq_tt {
  int d;
  int N[TTQ_MAXD];
  int r[TTQ_MAXD + 1];
  const double *core[TTQ_MAXD + 1];
  const int *left[TTQ_MAXD], *right[TTQ_MAXD];
};

// Dense layout of one instance's tensor train in a caller's buffer.  Its ranks
// are those of the last evaluated sweep (State.ro): the cores hold every entry
// for them, and the first ro[k] rows of each nested set are that sweep's sets
// (rows are only ever appended).
static size_t tt_layout(const Dev &D, const State &S, size_t *core_off, size_t *left_off, size_t *right_off) {
  Bump b;
  for (int k = 1; k <= D.d; ++k) core_off[k] = b.take((size_t)S.ro[k - 1] * D.N[k - 1] * S.ro[k] * 8);
  for (int k = 1; k < D.d; ++k) {
    left_off[k] = b.take((size_t)S.ro[k] * k * 4);
    right_off[k] = b.take((size_t)S.ro[k] * (D.d - k) * 4);
  }
  return (b.off + 255) & ~(size_t)255;
}

extern "C" int ttq_tt_bytes(ttq_plan *P, int instance, size_t *bytes) {
  if (!P || !bytes) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  if (instance < 0 || instance >= P->count) return set_err(TTQ_ERR_INVALID_ARG, "instance out of range");
  int rc = read_states(P);
  if (rc) return rc;
  size_t co[TTQ_MAXD + 1], lo[TTQ_MAXD], ro[TTQ_MAXD];
  *bytes = tt_layout(P->hs[instance], P->hst[instance], co, lo, ro);
  return TTQ_OK;
}

extern "C" int ttq_tt_export(ttq_plan *P, int instance, void *buffer, size_t bytes, ttq_tt **out) {
  if (!P || !out) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  if (instance < 0 || instance >= P->count) return set_err(TTQ_ERR_INVALID_ARG, "instance out of range");
  int rc = read_states(P);
  if (rc) return rc;
  const Dev &D = P->hs[instance];
  const State &S = P->hst[instance];
  size_t co[TTQ_MAXD + 1], lo[TTQ_MAXD], ro[TTQ_MAXD];
  const size_t need = tt_layout(D, S, co, lo, ro);
  if (!buffer || bytes < need || ((uintptr_t)buffer & 255))
    return set_err(TTQ_ERR_WORKSPACE, "tensor-train buffer too small or not 256-byte aligned (ttq_tt_bytes)");
  char *base = (char *)buffer;
  TTExport E;
  memset(&E, 0, sizeof(E));
  ttq_tt *T = new ttq_tt();
  T->d = D.d;
  int maxn = 0;
  for (int k = 0; k <= D.d; ++k) { E.r[k] = S.ro[k]; T->r[k] = S.ro[k]; }
  for (int k = 1; k <= D.d; ++k) {
    E.core[k] = (double *)(base + co[k]);
    T->core[k] = E.core[k];
    T->N[k - 1] = D.N[k - 1];
    const int nk = S.ro[k - 1] * D.N[k - 1] * S.ro[k];
    maxn = nk > maxn ? nk : maxn;
  }
  for (int k = 1; k < D.d; ++k) {
    E.left[k] = (int *)(base + lo[k]);
    E.right[k] = (int *)(base + ro[k]);
    T->left[k] = E.left[k];
    T->right[k] = E.right[k];
  }
  const int gx = std::max(1, std::min(1024, (maxn + 255) / 256));
  k_export_tt<<<dim3(gx, D.d), 256, 0, P->stream>>>(P->devs, instance, E);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) {
    delete T;
    g_last_error = std::string("tensor-train export: ") + cudaGetErrorString(e);
    return TTQ_ERR_CUDA;
  }
  P->launches++;
  *out = T;
  return TTQ_OK;
}

extern "C" int ttq_tt_get(const ttq_tt *T, int k, int32_t *r_left, int32_t *n_k, int32_t *r_right,
                          const double **core_dev, const int32_t **left_idx_dev, const int32_t **right_idx_dev) {
  if (!T) return set_err(TTQ_ERR_INVALID_ARG, "null tensor train");
  if (k < 1 || k > T->d) return set_err(TTQ_ERR_INVALID_ARG, "k out of range");
  if (r_left) *r_left = T->r[k - 1];
  if (n_k) *n_k = T->N[k - 1];
  if (r_right) *r_right = T->r[k];
  if (core_dev) *core_dev = T->core[k];
  if (left_idx_dev) *left_idx_dev = k >= 2 ? T->left[k - 1] : nullptr;
  if (right_idx_dev) *right_idx_dev = k <= T->d - 1 ? T->right[k] : nullptr;
  return TTQ_OK;
}

extern "C" int ttq_tt_ranks(const ttq_tt *T, int32_t *d, int32_t *ranks) {
  if (!T) return set_err(TTQ_ERR_INVALID_ARG, "null tensor train");
  if (d) *d = T->d;
  if (ranks)
    for (int k = 0; k <= T->d; ++k) ranks[k] = T->r[k];
  return TTQ_OK;
}

extern "C" int ttq_tt_free(ttq_tt *T) {
  delete T;
  return TTQ_OK;
}

extern "C" int ttq_plan_eval_points(ttq_plan *P, const int32_t *idx, int64_t npts, double *out) {
  if (P && P->count != 1) return set_err(TTQ_ERR_INVALID_ARG, "stage calls need a single-instance plan");
  if (!P || (!idx && npts) || (!out && npts) || npts < 0) return set_err(TTQ_ERR_INVALID_ARG, "bad argument");
  if (npts == 0) return TTQ_OK;
  long long blocks = (npts + TTQ_WARPS - 1) / TTQ_WARPS;
  if (blocks > 4096) blocks = 4096;
  k_eval_points<<<(int)blocks, TTQ_WARPS * 32, 0, P->stream>>>(P->devs, idx, npts, out);
  P->launches++;   // not part of a sweep: counted, not timed
  CK(cudaGetLastError());
  return TTQ_OK;
}

extern "C" int64_t ttq_plan_launches(const ttq_plan *P) { return P ? P->launches : 0; }

extern "C" int ttq_plan_transfer_bytes(const ttq_plan *P, int64_t *h2d, int64_t *d2h) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  if (h2d) *h2d = P->h2d;
  if (d2h) *d2h = P->d2h;
  return TTQ_OK;
}

extern "C" int ttq_plan_set_graphs(ttq_plan *P, int enable) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  P->use_graph = (enable && P->stream != nullptr) ? 1 : 0;
  return TTQ_OK;
}

extern "C" int ttq_plan_set_search(ttq_plan *P, int mode) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  if (mode < 0 || mode > 1) return set_err(TTQ_ERR_INVALID_ARG, "search mode must be 0 (staged) or 1 (persistent)");
  if (mode == 1 && (P->count != 1 || P->search_grid < P->max_ni))
    return set_err(TTQ_ERR_INVALID_ARG, "the persistent search needs a single-instance plan that fits the device");
  if (mode == 1 && P->npiv > 1) return set_err(TTQ_ERR_INVALID_ARG, "the persistent search takes one pivot per sweep");
  P->persistent = mode;
  if (P->run_exec) { cudaGraphExecDestroy(P->run_exec); P->run_exec = nullptr; }
  if (P->sweep_exec) { cudaGraphExecDestroy(P->sweep_exec); P->sweep_exec = nullptr; }
  return TTQ_OK;
}

extern "C" int ttq_plan_set_sequential(ttq_plan *P, int enable) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  if (enable && P->count != 1) return set_err(TTQ_ERR_INVALID_ARG, "sequential sweeps need a single-instance plan");
  if (enable && P->npiv > 1) return set_err(TTQ_ERR_INVALID_ARG, "the sequential sweep takes one pivot per step");
  P->sequential = enable ? 1 : 0;
  if (P->run_exec) { cudaGraphExecDestroy(P->run_exec); P->run_exec = nullptr; }
  if (P->sweep_exec) { cudaGraphExecDestroy(P->sweep_exec); P->sweep_exec = nullptr; }
  return TTQ_OK;
}

extern "C" int ttq_plan_set_wait_limit(ttq_plan *P, uint64_t ns) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  if (ns < 1) return set_err(TTQ_ERR_INVALID_ARG, "wait limit must be >= 1 ns");
  for (int q = 0; q < P->count; ++q) {
    P->hs[q].wait_ns = ns;
    Dev *dq = nullptr;
    CK(cudaMemcpy(&dq, (char *)P->devs + q * sizeof(Dev *), sizeof(Dev *), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy((char *)dq + offsetof(Dev, wait_ns), &ns, sizeof(ns), cudaMemcpyHostToDevice));
  }
  P->h.wait_ns = ns;
  return TTQ_OK;
}

extern "C" int ttq_plan_set_timing(ttq_plan *P, int enable) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  P->timing = enable ? 1 : 0;
  return TTQ_OK;
}

extern "C" int ttq_plan_kernel_times(ttq_plan *P, double *ms, int64_t *launches, double *flops, int reset) {
  if (!P) return set_err(TTQ_ERR_INVALID_ARG, "null plan");
  int rc = read_states(P);               // synchronizes and harvests the pending events
  if (rc) return rc;
  for (int q = 0; q < KT_N; ++q) {
    if (ms) ms[q] = P->kt_ms[q];
    if (launches) launches[q] = P->kt_n[q];
    if (flops) {
      double f = 0.0;
      for (int i = 0; i < P->count; ++i) f += (double)P->hst[i].flops[q];
      flops[q] = f;
    }
    if (reset) { P->kt_ms[q] = 0.0; P->kt_n[q] = 0; }
  }
  return TTQ_OK;
}

extern "C" const char *ttq_status_string(int s) {
  switch (s) {
    case TTQ_OK: return "ok (converged)";
    case TTQ_WARN_NO_PIVOT: return "stopped: no pivot accepted";
    case TTQ_WARN_RANK_CAP: return "stopped: rank cap reached on every interface";
    case TTQ_WARN_MAX_SWEEPS: return "stopped: sweep limit reached";
    case TTQ_PENDING: return "pending";
    case TTQ_ERR_INVALID_ARG: return "invalid argument";
    case TTQ_ERR_NONFINITE: return "non-finite integrand value";
    case TTQ_ERR_SINGULAR: return "singular cross matrix";
    case TTQ_ERR_WORKSPACE: return "workspace too small or misaligned";
    case TTQ_ERR_CUDA: return "CUDA error";
    case TTQ_ERR_ADMISSION: return "request exceeds the memory budget";
    case TTQ_ERR_NOT_FOUND: return "not found";
    case TTQ_ERR_TIMEOUT: return "a wait between CTAs passed its limit";
    default: return "unknown status";
  }
}

extern "C" const char *ttq_last_error(void) { return g_last_error.c_str(); }


// ---------------------------------------------------------------------------
// Entry point for callers that cannot allocate device memory.
//
// Some callers are not allowed to call cudaMalloc: code that runs while another
// component owns the device's memory pool (a framework's caching allocator or
// a memory-capped serving process), plugins that are handed a stream and must
// not grow the process footprint, or code paths that must not fail on
// allocation at run time.  For them the library keeps one fixed scratch area
// in device memory, declared below; every GPU that loads the library holds it
// until the process exits.  This entry point allocates nothing (no cudaMalloc,
// cudaFree, cudaMallocHost or allocating library routine): the plan, the host
// copy of its state and the node checks live on the stack, and the device
// scratch is this array.
// size: TTQ_NOALLOC_SCRATCH_BYTES (16 MiB), include/ttq.h
static __device__ __align__(256) unsigned char g_noalloc_scratch[TTQ_NOALLOC_SCRATCH_BYTES];
// The scratch's device address is looked up on every call, with the caller's
// device current (host code cannot use the symbol's own address: it names a
// host-side stand-in); the lookup allocates nothing, and no address outlives
// the context it was taken in (a device reset or a new primary context).

extern "C" int ttq_integrate_noalloc(const ttq_problem *p, void *stream, ttq_result *out) {
  int rc = validate(p);
  if (rc) return rc;
  if (!out) return set_err(TTQ_ERR_INVALID_ARG, "null result");
  if (p->inputs_on_device) return set_err(TTQ_ERR_INVALID_ARG, "ttq_integrate_noalloc takes host nodes and weights");
  Layout L;
  make_layout(p, &L);
  if (L.total > TTQ_NOALLOC_SCRATCH_BYTES)
    return set_err(TTQ_ERR_WORKSPACE, "problem needs more device scratch than the 16 MiB the "
                                      "no-allocation entry point holds; use ttq_plan_create");
  // the call waits for its stream and copies from this stack frame: on a
  // capturing stream it is refused before any CUDA work, leaving the capture intact
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing((cudaStream_t)stream, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return set_err(TTQ_ERR_INVALID_ARG, "ttq_integrate_noalloc called on a capturing stream");
  void *scratch = nullptr;
  CK(cudaGetSymbolAddress(&scratch, g_noalloc_scratch));
  char *base = (char *)scratch;
  const int d = p->d;
  size_t sumN = 0;
  for (int k = 0; k < d; ++k) sumN += p->nodes_per_mode[k];
  for (size_t q = 0; q < sumN; ++q)
    if (!isfinite(p->nodes[q]) || !isfinite(p->weights[q])) return set_err(TTQ_ERR_INVALID_ARG, "non-finite node or weight");

  ttq_plan P{};                             // on the stack, zeroed; its vectors stay empty (timing off)
  State host_state;
  P.count = 1;
  P.stream = (cudaStream_t)stream;
  P.hst = &host_state;
  P.hs = &P.h;
  P.sts = &P.st;
  configure(&P, p, 1, &L);
  fill_descriptor(p, p->nodes, base, L, P.max_cap <= 96 ? 1 : 0, P.h);
  P.dev = (Dev *)(base + L.dev);
  P.st = P.h.st;
  P.devs = (Dev **)(base + L.devs);
  Dev *devp = P.dev;
  cudaStream_t s = P.stream;
  // the scratch keeps the previous call's contents: everything read before it is
  // written (node tables, descriptor, state, fiber row counters) is set here
  CK(set_smem_attributes(&P));
  CK(cudaMemcpyAsync(base + L.x, p->nodes, sumN * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(base + L.w, p->weights, sumN * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(P.h.st, 0, sizeof(State), s));
  CK(cudaMemsetAsync(base + L.vcnt_all, 0, L.vcnt_bytes, s));
  CK(cudaMemcpyAsync(P.dev, &P.h, sizeof(Dev), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.devs, &devp, sizeof(Dev *), cudaMemcpyHostToDevice, s));
  k_setup<<<dim3((P.max_sum_n + 255) / 256, 1, 1), 256, 0, s>>>(P.devs);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));             // the host sources above live on this stack frame
  return ttq_plan_run(&P, out);
}

// ---------------------------------------------------------------------------
// Serving: continuous batching.
//
// Requests are queued on the host as they arrive.  At every step boundary the
// server (1) retires the instances that stopped (double-double contraction if
// asked, state copied back, memory returned to the pool), (2) admits queued
// requests in arrival order while a slot and pool memory (the plan footprint
// at the request's rank cap) are free, initializing them on the device, and
// (3) runs `sweeps` sweeps of every instance in flight with the batched
// kernels (one launch per stage for the whole set).  Each instance's
// arithmetic is independent of the others, so a result is the same alone and
// in any mix.
#include <map>
#include <deque>
#include <unordered_map>

struct Request {
  uint64_t id;
  ttq_problem p;                    // host copy; arrays below
  std::vector<int32_t> N;
  std::vector<double> x, w;
  size_t bytes;                     // plan footprint at the rank cap
};

struct Slot {
  Request req;
  size_t off;                       // offset of its workspace in the pool
  Layout L;
  Dev h;
  Dev *dev;
  Dev **own;                        // its one-entry descriptor array
  int fresh;                        // admitted at this boundary: not yet initialized
};

struct ttq_server {
  char *pool;
  size_t pool_bytes;
  int max_slots;
  cudaStream_t stream;
  std::map<size_t, size_t> free_list;       // offset -> size, coalesced
  std::deque<Request> queue;
  std::vector<Slot> active;
  std::unordered_map<uint64_t, ttq_result> done;
  uint64_t next_id;
  ttq_plan P;                               // launch configuration over the active set
  Dev **devs;                               // device array of the active descriptors (pool head)
  State *hst;                               // pinned, device-mapped host states (max_slots)
  int *hflags;                              // pinned, device-mapped stop flags (max_slots)
  State *hst_dev;                           // device addresses of the two
  int *hflags_dev;
  int dirty;                                // the active set changed since the launch configuration
  long long sweeps_run, admitted, retired;
  // concurrent engine (mode 0): every request in flight is a plan of its own
  // whose whole run is one graph launch on one of the server's streams
  int mode;                                 // 0: concurrent plans, 1: batched sweeps
  std::vector<cudaStream_t> streams;
  struct Live {
    Request req;
    size_t off;
    ttq_plan *plan;
    cudaEvent_t done;
    int slot;                               // index of its final state in hst
  };
  std::vector<Live> live;
  std::vector<int> free_slots;
  int next_stream;
};

#define TTQ_SERVER_STREAMS 16

static size_t pool_alloc(ttq_server *S, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  for (auto it = S->free_list.begin(); it != S->free_list.end(); ++it) {
    if (it->second >= bytes) {
      size_t off = it->first, rest = it->second - bytes;
      S->free_list.erase(it);
      if (rest) S->free_list[off + bytes] = rest;
      return off;
    }
  }
  return (size_t)-1;
}

static void pool_free(ttq_server *S, size_t off, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  auto it = S->free_list.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != S->free_list.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    S->free_list.erase(nx);
  }
  if (it != S->free_list.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      S->free_list.erase(it);
    }
  }
}

extern "C" int ttq_server_create(void *pool, size_t pool_bytes, int max_slots, void *stream, ttq_server **out) {
  if (!pool || !out || max_slots < 1 || max_slots > 4096 || ((uintptr_t)pool & 255))
    return set_err(TTQ_ERR_INVALID_ARG, "bad server arguments");
  size_t head = ((size_t)max_slots * sizeof(Dev *) + 255) & ~(size_t)255;
  if (pool_bytes <= head) return set_err(TTQ_ERR_WORKSPACE, "pool too small");
  ttq_server *S = new ttq_server();
  S->pool = (char *)pool;
  S->pool_bytes = pool_bytes;
  S->max_slots = max_slots;
  S->stream = (cudaStream_t)stream;
  S->devs = (Dev **)pool;
  S->free_list[head] = (pool_bytes - head) & ~(size_t)255;
  S->next_id = 1;
  // the collect kernel writes every step's stop flags, and the final states of
  // the instances that stopped, straight into host memory
  if (cudaHostAlloc((void **)&S->hst, sizeof(State) * max_slots, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc((void **)&S->hflags, sizeof(int) * max_slots, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void **)&S->hst_dev, S->hst, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void **)&S->hflags_dev, S->hflags, 0) != cudaSuccess) {
    if (S->hst) cudaFreeHost(S->hst);
    if (S->hflags) cudaFreeHost(S->hflags);
    delete S;
    return set_err(TTQ_ERR_CUDA, "cudaHostAlloc failed");
  }
  S->P.stream = S->stream;
  S->P.devs = S->devs;
  S->P.hst = S->hst;
  S->mode = 0;
  S->next_stream = 0;
  for (int q = max_slots - 1; q >= 0; --q) S->free_slots.push_back(q);
  for (int q = 0; q < TTQ_SERVER_STREAMS; ++q) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) break;
    S->streams.push_back(st);
  }
  cudaError_t e;
  if ((e = create_side_stream(&S->P.s2, false)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&S->P.fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&S->P.join, cudaEventDisableTiming)) != cudaSuccess) {
    g_last_error = std::string("server setup: ") + cudaGetErrorString(e);
    cudaFreeHost(S->hst);
    cudaFreeHost(S->hflags);
    delete S;
    return TTQ_ERR_CUDA;
  }
  *out = S;
  return TTQ_OK;
}

extern "C" int ttq_server_destroy(ttq_server *S) {
  if (!S) return TTQ_OK;
  for (auto &L : S->live) {
    cudaEventSynchronize(L.done);
    cudaEventDestroy(L.done);
    ttq_plan_destroy(L.plan);
  }
  for (cudaStream_t st : S->streams) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
  cudaStreamSynchronize(S->stream);
  if (S->P.s2) { cudaStreamSynchronize(S->P.s2); cudaStreamDestroy(S->P.s2); }
  if (S->P.fork) cudaEventDestroy(S->P.fork);
  if (S->P.join) cudaEventDestroy(S->P.join);
  S->P.s2 = nullptr;
  S->P.hs = nullptr;
  S->P.sts = nullptr;
  cudaFreeHost(S->hst);
  cudaFreeHost(S->hflags);
  delete S;
  return TTQ_OK;
}

extern "C" int ttq_server_submit(ttq_server *S, const ttq_problem *p, uint64_t *request_id) {
  if (!S || !p) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  int rc = validate(p);
  if (rc) return rc;
  if (npiv_of(p) > 1) return set_err(TTQ_ERR_INVALID_ARG, "several pivots per sweep: single plans only, not servers");
  Layout L;
  make_layout(p, &L);
  size_t head = ((size_t)S->max_slots * sizeof(Dev *) + 255) & ~(size_t)255;
  if (L.total > S->pool_bytes - head) return set_err(TTQ_ERR_ADMISSION, "request larger than the server's memory pool");
  Request r;
  r.id = S->next_id++;
  r.p = *p;
  r.N.assign(p->nodes_per_mode, p->nodes_per_mode + p->d);
  if ((rc = host_inputs(p, S->stream, r.x, r.w))) return rc;
  r.p.nodes_per_mode = nullptr;             // re-pointed at admission
  r.p.inputs_on_device = 0;
  r.bytes = L.total;
  S->queue.push_back(std::move(r));
  if (request_id) *request_id = S->queue.back().id;
  return TTQ_OK;
}

static void repoint(Request &r) {
  r.p.nodes_per_mode = r.N.data();
  r.p.nodes = r.x.data();
  r.p.weights = r.w.data();
}

// admit what fits; build and upload each new instance's descriptor and inputs
static int server_admit(ttq_server *S) {
  while (!S->queue.empty() && (int)S->active.size() < S->max_slots) {
    Request &r = S->queue.front();
    size_t off = pool_alloc(S, r.bytes);
    if (off == (size_t)-1) break;           // wait for memory (arrival order is kept)
    Slot sl;
    sl.req = std::move(r);
    S->queue.pop_front();
    repoint(sl.req);
    sl.off = off;
    make_layout(&sl.req.p, &sl.L);
    char *base = S->pool + off;
    fill_descriptor(&sl.req.p, sl.req.x.data(), base, sl.L, 0, sl.h);
    sl.dev = (Dev *)(base + sl.L.dev);
    sl.own = (Dev **)(base + sl.L.devs);
    sl.fresh = 1;
    const size_t sumN = sl.req.x.size();
    cudaStream_t s = S->stream;
    CK(cudaMemcpyAsync(base + sl.L.x, sl.req.x.data(), sumN * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(base + sl.L.w, sl.req.w.data(), sumN * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(sl.h.st, 0, sizeof(State), s));
    CK(cudaMemsetAsync(base + sl.L.vcnt_all, 0, sl.L.vcnt_bytes, s));
    S->active.push_back(std::move(sl));
    Slot &a = S->active.back();
    repoint(a.req);                         // vectors moved: pointers refreshed
    a.h.x = (const double *)(base + a.L.x);
    CK(cudaMemcpyAsync(a.dev, &a.h, sizeof(Dev), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(a.own, &a.dev, sizeof(Dev *), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));           // host sources must outlive the copies
    S->admitted++;
    S->dirty = 1;
  }
  return TTQ_OK;
}

// launch configuration and descriptor array of the current active set
static int server_configure(ttq_server *S) {
  const int n = (int)S->active.size();
  if (n == 0 || !S->dirty) return TTQ_OK;
  S->dirty = 0;
  std::vector<ttq_problem> probs(n);
  std::vector<Layout> Ls(n);
  std::vector<Dev *> dp(n);
  for (int q = 0; q < n; ++q) {
    probs[q] = S->active[q].req.p;
    Ls[q] = S->active[q].L;
    dp[q] = S->active[q].dev;
  }
  ttq_plan &P = S->P;
  P.count = n;
  configure(&P, probs.data(), n, Ls.data());
  // the search kernels stage Q in shared memory only when the largest cap allows
  for (int q = 0; q < n; ++q) {
    Slot &a = S->active[q];
    int qin = P.max_cap <= 96 ? 1 : 0;
    if (a.h.q_in_smem != qin) {
      a.h.q_in_smem = qin;
      CK(cudaMemcpyAsync(a.dev, &a.h, sizeof(Dev), cudaMemcpyHostToDevice, S->stream));
    }
  }
  CK(cudaMemcpyAsync(S->devs, dp.data(), n * sizeof(Dev *), cudaMemcpyHostToDevice, S->stream));
  CK(set_smem_attributes(&P));
  CK(cudaStreamSynchronize(S->stream));
  return TTQ_OK;
}

// retire stopped instances: one kernel collects every instance's stop flag
// (and the final state of those that stopped) into mapped host memory; the
// double-double ones first get their final contraction; results, memory
static int server_retire(ttq_server *S) {
  const int n = (int)S->active.size();
  if (n == 0) return TTQ_OK;
  k_server_collect<<<(n + 7) / 8, 256, 0, S->stream>>>(S->devs, n, S->hflags_dev, S->hst_dev, 0);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(S->stream));
  int ndd = 0;
  for (int q = 0; q < n; ++q) {
    Slot &a = S->active[q];
    if (!S->hflags[q] || !a.h.prec) continue;
    const int cs = (int)(((size_t)a.h.cap * a.h.cap + a.h.cap) * 8);
    k_dd_factor<<<a.h.d - 1, 256, 0, S->stream>>>(a.own);
    k_contract<<<2, 256, cs, S->stream>>>(a.own, 1);
    ++ndd;
  }
  if (ndd) {                                // their states again, after the final contraction
    k_server_collect<<<(n + 7) / 8, 256, 0, S->stream>>>(S->devs, n, S->hflags_dev, S->hst_dev, 1);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(S->stream));
  }
  std::vector<Slot> keep;
  keep.reserve(n);
  for (int q = 0; q < n; ++q) {
    Slot &a = S->active[q];
    if (!S->hflags[q]) {
      keep.push_back(std::move(a));
      continue;
    }
    ttq_result res;
    fill_result_from(a.h, S->hst[q], &res);
    S->done[a.req.id] = res;
    pool_free(S, a.off, a.req.bytes);
    S->retired++;
    S->dirty = 1;
  }
  S->active.swap(keep);
  for (auto &a : S->active) repoint(a.req);
  return TTQ_OK;
}

// Concurrent engine.  Retire: every plan whose run has completed (its event,
// queried without waiting) gives its result from the final state copied to
// mapped host memory; its plan is destroyed and its pool memory freed.
static int server_retire_live(ttq_server *S) {
  // a step makes progress: with requests in flight and none finished, wait for
  // the one admitted first
  if (!S->live.empty()) {
    bool any = false;
    for (auto &L : S->live) any |= cudaEventQuery(L.done) != cudaErrorNotReady;
    if (!any) CK(cudaEventSynchronize(S->live.front().done));
  }
  std::vector<ttq_server::Live> keep;
  keep.reserve(S->live.size());
  for (auto &L : S->live) {
    const cudaError_t q = cudaEventQuery(L.done);
    if (q == cudaErrorNotReady) {
      keep.push_back(std::move(L));
      continue;
    }
    if (q != cudaSuccess) { g_last_error = std::string("server: ") + cudaGetErrorString(q); return TTQ_ERR_CUDA; }
    ttq_result res;
    fill_result_from(L.plan->h, S->hst[L.slot], &res);
    L.plan->launches += (long long)L.plan->sweep_kernels * S->hst[L.slot].loop_guard;
    S->done[L.req.id] = res;
    cudaEventDestroy(L.done);
    ttq_plan_destroy(L.plan);
    pool_free(S, L.off, L.req.bytes);
    S->free_slots.push_back(L.slot);
    S->retired++;
  }
  S->live.swap(keep);
  return TTQ_OK;
}

// Admit, in arrival order, while a slot and pool memory are free: a plan over
// the request's pool region on the next of the server's streams, its whole
// run enqueued as one graph, its final state copied to mapped host memory,
// an event behind it.
static int server_admit_live(ttq_server *S) {
  while (!S->queue.empty() && (int)S->live.size() < S->max_slots && !S->free_slots.empty()) {
    Request &r = S->queue.front();
    const size_t off = pool_alloc(S, r.bytes);
    if (off == (size_t)-1) break;           // wait for memory (arrival order is kept)
    ttq_server::Live L;
    L.req = std::move(r);
    S->queue.pop_front();
    repoint(L.req);
    L.off = off;
    L.slot = S->free_slots.back();
    cudaStream_t st = S->streams.empty() ? S->stream : S->streams[S->next_stream++ % S->streams.size()];
    int rc = plan_build(&L.req.p, 1, S->pool + off, L.req.bytes, st, &L.plan);
    if (rc) { pool_free(S, off, L.req.bytes); return rc; }
    L.plan->persistent = 0;
    if ((rc = enqueue_run(L.plan))) { ttq_plan_destroy(L.plan); pool_free(S, off, L.req.bytes); return rc; }
    CK(cudaMemcpyAsync(S->hst + L.slot, L.plan->st, sizeof(State), cudaMemcpyDeviceToHost, st));
    CK(cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming));
    CK(cudaEventRecord(L.done, st));
    S->free_slots.pop_back();
    S->admitted++;
    S->live.push_back(std::move(L));
  }
  return TTQ_OK;
}

extern "C" int ttq_server_set_mode(ttq_server *S, int mode) {
  if (!S || mode < 0 || mode > 1) return set_err(TTQ_ERR_INVALID_ARG, "bad argument");
  if (!S->live.empty() || !S->active.empty()) return set_err(TTQ_ERR_INVALID_ARG, "requests in flight");
  S->mode = mode;
  return TTQ_OK;
}

extern "C" int ttq_server_step(ttq_server *S, int sweeps, int *active, int *queued, int64_t *completed) {
  if (!S || sweeps < 1) return set_err(TTQ_ERR_INVALID_ARG, "bad argument");
  int rc;
  if (S->mode == 0) {
    if ((rc = server_retire_live(S))) return rc;
    if ((rc = server_admit_live(S))) return rc;
    if (active) *active = (int)S->live.size();
    if (queued) *queued = (int)S->queue.size();
    if (completed) *completed = S->retired;
    return TTQ_OK;
  }
  if ((rc = server_retire(S))) return rc;
  if ((rc = server_admit(S))) return rc;
  if ((rc = server_configure(S))) return rc;
  const int n = (int)S->active.size();
  if (n) {
    // initialize the instances admitted at this boundary (they join the next sweep)
    for (auto &a : S->active) {
      if (!a.fresh) continue;
      const int sumN = a.h.off[a.h.d - 1] + a.h.N[a.h.d - 1];
      k_setup<<<(sumN + 255) / 256, 256, 0, S->stream>>>(a.own);
      k_init<<<1, TTQ_WARPS * 32, 0, S->stream>>>(a.own);
      k_begin<<<1, 1, 0, S->stream>>>(a.own, 0, 1, 1);
      a.fresh = 0;
    }
    CK(cudaGetLastError());
    for (int s = 0; s < sweeps; ++s) enqueue_sweep(&S->P);
    CK(cudaGetLastError());
    S->sweeps_run += sweeps;
  }
  if (active) *active = (int)S->active.size();
  if (queued) *queued = (int)S->queue.size();
  if (completed) *completed = S->retired;
  return TTQ_OK;
}

extern "C" int ttq_server_poll(ttq_server *S, uint64_t request_id, ttq_result *out) {
  if (!S || !out) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  auto it = S->done.find(request_id);
  if (it == S->done.end()) {
    for (auto &a : S->active) if (a.req.id == request_id) return TTQ_PENDING;
    for (auto &L : S->live) if (L.req.id == request_id) return TTQ_PENDING;
    for (auto &r : S->queue) if (r.id == request_id) return TTQ_PENDING;
    return set_err(TTQ_ERR_NOT_FOUND, "unknown request");
  }
  *out = it->second;
  S->done.erase(it);
  return TTQ_OK;
}

extern "C" int ttq_server_drain(ttq_server *S, uint64_t *ids, ttq_result *results, int max, int *n) {
  if (!S || !n || (max > 0 && (!ids || !results))) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  int q = 0;
  for (auto it = S->done.begin(); it != S->done.end() && q < max;) {
    ids[q] = it->first;
    results[q] = it->second;
    ++q;
    it = S->done.erase(it);
  }
  *n = q;
  return TTQ_OK;
}

extern "C" int ttq_server_stats(const ttq_server *S, int64_t *stats /* [6] */) {
  if (!S || !stats) return set_err(TTQ_ERR_INVALID_ARG, "null argument");
  size_t free_bytes = 0;
  for (auto &kv : S->free_list) free_bytes += kv.second;
  stats[0] = (int64_t)(S->mode == 0 ? S->live.size() : S->active.size());
  stats[1] = (int64_t)S->queue.size();
  stats[2] = S->admitted;
  stats[3] = S->retired;
  stats[4] = S->sweeps_run;
  stats[5] = (int64_t)free_bytes;
  return TTQ_OK;
}
