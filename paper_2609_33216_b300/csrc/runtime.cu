// Host runtime of the symhss library: trees and proxy rings, height-by-height
// scheduling of the compression (Sec. 4.1), factorisation and solve (Sec. 4.2),
// device memory, and the C ABI declared in include/symhss.h.
//
// A handle holds one or more independent scatterers ("problems"), each with its
// own curve, wavenumbers, materials and tree.  Work is scheduled by tree height
// (counted from the leaves): the boxes of every problem at height t are processed
// together, one launch per kernel, so a batch of uneven scatterers costs no more
// launches than its tallest tree.  A problem's root sits at height = its depth.
//
// Tree (Sec. 4.1, Theorem 1 setting): a binary tree over the node index order;
// box [b, e) splits into [b, b + (e - b)/2) and the rest; all leaves at depth
// L = ceil(log2(N / leaf)).  Box centre = mean of its nodes, radius rho = largest
// node distance from the centre; proxy ring radius R = proxy_factor * rho with
// P = max(nproxy, 8 ceil((2 max(k0, k1) R + 32) / 8)) equispaced points, outward
// radial normals and weights 2 pi R / P.
//
// Compression of a box: its active unknowns are its nodes (leaf) or its children's
// skeletons.  M_R rows are the near (point, equation) pairs -- active rows of other
// boxes of the same problem and level strictly inside the proxy ring -- ordered
// [equation 1 rows; equation 2 rows], then the P proxy points for equation 1 and
// for equation 2; its columns are the box's active flux unknowns then trace
// unknowns.  One column ID per half (symmetric mode, Eq. low-rank_R: L = R^T).
// The baseline also builds M_L^T (the box's active equations against near active
// unknowns and proxy sources) and row-IDs each half; per half both ranks are
// raised to their maximum so that R D^{-1} L is square.
#include <algorithm>
#include <initializer_list>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

namespace symhss {

// ---- growable device buffer -------------------------------------------------------
// A handle's device-memory budget (symhss_set_memory_limit): the bytes its growable buffers
// hold.  While one of the handle's calls runs, g_budget points at it; a buffer remembers
// the budget it was allocated under and returns its bytes on release.
struct Budget {
  long long limit = 0;  // <= 0: none
  long long used = 0;
};
thread_local Budget* g_budget = nullptr;

struct BudgetScope {
  Budget* saved;
  explicit BudgetScope(Budget* b) : saved(g_budget) { g_budget = b; }
  ~BudgetScope() { g_budget = saved; }
};

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  Budget* bud = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), cap(o.cap), bud(o.bud) { o.p = nullptr; o.cap = 0; o.bud = nullptr; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; cap = o.cap; bud = o.bud;
      o.p = nullptr; o.cap = 0; o.bud = nullptr;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      cudaFree(p);
      if (bud) bud->used -= (long long)cap;
    }
    p = nullptr;
    cap = 0;
    bud = nullptr;
  }
  // grow to at least `bytes` (contents are not preserved on growth); beyond the current
  // call's budget this fails as an out-of-memory allocation, without calling cudaMalloc
  cudaError_t ensure(size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (bytes <= cap) return cudaSuccess;
    release();
    Budget* b = g_budget;
    if (b && b->limit > 0 && b->used + (long long)bytes > b->limit) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) { p = nullptr; return e; }
    cap = bytes;
    bud = b;
    if (bud) bud->used += (long long)bytes;
    return cudaSuccess;
  }
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

// pack several host arrays into one device buffer (one copy); returns offsets
struct Packer {
  std::vector<char> host;
  size_t add(const void* src, size_t bytes) {
    size_t off = (host.size() + 255) & ~size_t(255);
    host.resize(off + bytes);
    if (bytes && src) std::memcpy(host.data() + off, src, bytes);
    if (bytes && !src) std::memset(host.data() + off, 0, bytes);
    return off;
  }
  template <class T> size_t add(const std::vector<T>& v) { return add(v.data(), v.size() * sizeof(T)); }
  cudaError_t upload(DevBuf& buf, cudaStream_t s) {
    cudaError_t e = buf.ensure(host.size());
    if (e != cudaSuccess) return e;
    if (host.empty()) return cudaSuccess;
    return cudaMemcpyAsync(buf.p, host.data(), host.size(), cudaMemcpyHostToDevice, s);
  }
};

struct HBox {
  int begin = 0, end = 0;  // node range in the handle's concatenated node order
  double cx = 0, cy = 0, rho = 0, R = 0;
  int P = 0;
  int proxy0 = 0;  // first proxy point in the point table
  int m_near = 0;  // near rows of M_R (both equations)
  int child[2] = {-1, -1};
  std::vector<int> act[2], actrow[2];
  int rank[2] = {0, 0}, rrank[2] = {0, 0};
  std::vector<int> perm[2], rperm[2];
  long long t_off[2] = {0, 0}, rt_off[2] = {0, 0};  // into the height's T buffer
  // factor
  int size = 0;      // diagonal-block order
  int k = 0;         // rank[0] + rank[1]
  long long d_off = 0, piv_off = 0, x_off = 0, rx_off = 0;
  long long q_off[2] = {0, 0}, rq_off[2] = {0, 0};
  long long rxpiv_off = 0;
  // solve
  long long g_off = 0, ft_off = 0;
};

// One scatterer of the handle.
struct Problem {
  symhss_params prm{};
  int n = 0, depth = 0;
  int node0 = 0;                           // first node in the concatenated node order
  long long vec0 = 0;                      // first row of its [eq1; eq2] block in batch vectors
  std::vector<std::vector<HBox>> levels;   // boxes of levels 0 .. depth
  int lvl_max_rank[SYMHSS_MAX_LEVELS][2] = {};  // largest column-ID rank per level and part
};

// Device buffers of all boxes at one tree height (over every problem of the handle).
struct Height {
  // compress
  DevBuf mr, tbuf, permbuf, rankbuf, refbuf, clists, idjobs, slices, skmeta;
  // factor
  DevBuf D, piv, rxpiv, info, X, RX, At, qbuf, flists, lujobs, cjobs;
  DevBuf perm, rxperm;           // the LUs' row permutations (kept by the LU, read by the solves)
  DevBuf Dop;                    // the assembled diagonal blocks (FP64), kept for the matvec
  DevBuf D32, X32, RX32, At32;   // complex64 work of the mixed-precision factorisation
  // solve
  DevBuf G, FT, TMP, slists;
  DevBuf chkmeta, chkg;          // exact residual checks of sketched IDs (proposer mode)
  DevBuf chkimg;                 // their tensor-core product scratch (compression stream)
  DevBuf zimg;                   // tensor-core product scratch of the factorisation stream
  DevBuf dinv;                   // inverses of the diagonal blocks of the blocked solves
  // matvec
  DevBuf XV, XS, ZV, YS, YV, mlists;
  std::vector<int> h_rank;
};

// A box at some height: problem p, level l, index b in that level.
struct BoxRef {
  int p, l, b;
  HBox* bx;
};

}  // namespace symhss

struct symhss_s {
  symhss_params prm{};                            // shared parameters (problem 0's)
  std::vector<symhss::Problem> probs;
  int ntot = 0;                                   // nodes over all problems
  int maxdepth = 0;
  std::vector<double> hx, hy, hnx, hny, hw, hk;  // concatenated node arrays on the host
  int npts = 0;                                   // nodes + proxy points
  symhss::DevBuf pts;                             // point table (7 arrays)
  symhss::DevBuf kps;                             // KernelParams per problem
  symhss::DevBuf waves;                           // WaveJob per problem
  int max_n = 0;                                  // largest problem
  symhss::DevBuf status;
  std::vector<symhss::Height> heights;            // 0 .. maxdepth
  bool compressed = false, factored = false;
  symhss::DevBuf xin, xout;                       // host-buffer solve staging
  cudaEvent_t ev[8] = {};
  // per-launch device timing: events recorded around each launch on the caller's stream
  std::vector<cudaEvent_t> evpool;
  size_t evnext = 0;
  struct Mark { int cls, e0, e1; double work; };
  std::vector<Mark> marks;
  symhss_stats_t st{};
  cudaError_t last_cuda = cudaSuccess;
  std::vector<int> mark;                          // host scratch (size npts)
  symhss_tuning tune = {0, 256, 0, 16, 16, 1, 16, {0}};  // launch tuning (symhss_set_tuning)
  symhss_mlp_s* mlp = nullptr;                    // attached proposer (not owned)
  double prop_margin = 1.15;
  symhss::DevBuf featjobs, feats, mlpout, chkjobs, chkratio;
  int refine_steps = 2;                           // SYMHSS_MIXED solves
  cudaStream_t cstream = nullptr;                 // high-priority stream of the pipelined build
  symhss::DevBuf rres, rcor, rtmp;                // refinement vectors
  int rank_limit = 0;                             // symhss_set_rank_limit (<= 0: none)
  symhss::Budget budget;                          // symhss_set_memory_limit
};

namespace symhss {

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

int cuda_fail(symhss_s* h, cudaError_t e) {
  if (h) h->last_cuda = e;
  return e == cudaErrorMemoryAllocation ? SYMHSS_ERR_NOMEM : SYMHSS_ERR_CUDA;
}
#define CK(call)                                   \
  do {                                             \
    cudaError_t _e = (call);                       \
    if (_e != cudaSuccess) return cuda_fail(h, _e); \
  } while (0)

// Record an event before a launch; returns its pool index or -1 (timing skipped).
int prof_begin(symhss_s* h, cudaStream_t s) {
  if (h->evnext >= h->evpool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    h->evpool.push_back(e);
  }
  const int i = (int)h->evnext++;
  if (cudaEventRecord(h->evpool[i], s) != cudaSuccess) return -1;
  return i;
}
void prof_end(symhss_s* h, cudaStream_t s, int cls, int e0, double work) {
  if (e0 < 0) return;
  const int e1 = prof_begin(h, s);
  if (e1 < 0) return;
  h->marks.push_back({cls, e0, e1, work});
}
// After a stream synchronisation: fold the recorded launches into the statistics.
// Marks whose end event has not completed yet (work still running on another stream of
// a pipelined build) are kept, and the event pool is reused only once no mark is pending.
void prof_collect(symhss_s* h) {
  std::vector<symhss_s::Mark> pending;
  for (const auto& m : h->marks) {
    if (cudaEventQuery(h->evpool[m.e1]) == cudaErrorNotReady) {
      pending.push_back(m);
      continue;
    }
    cudaGetLastError();
    float ms = 0;
    if (cudaEventElapsedTime(&ms, h->evpool[m.e0], h->evpool[m.e1]) == cudaSuccess) h->st.kernel_ms[m.cls] += ms;
    else cudaGetLastError();
    h->st.kernel_launches[m.cls] += 1;
    h->st.kernel_work[m.cls] += m.work;
  }
  h->marks.swap(pending);
  if (h->marks.empty()) h->evnext = 0;
}
#define TIMED(cls, work, call)                     \
  do {                                             \
    const int _e0 = prof_begin(h, s);              \
    CK(call);                                      \
    prof_end(h, s, (cls), _e0, (work));            \
  } while (0)

double id_flops(int m, int n, int r) {
  // Householder application (16 real flops per trailing entry and step) + T = R11^{-1} R12
  double f = 0;
  for (int k = 0; k < r; ++k) f += 16.0 * (double)(m - k) * (double)(n - k - 1);
  return f + 4.0 * (double)r * r * (n - r);
}

bool finite_all(const std::vector<double>& v) {
  for (double a : v)
    if (!std::isfinite(a)) return false;
  return true;
}

PointTable table_of(const symhss_s* h) {
  const double* base = h->pts.as<double>();
  const size_t np = (size_t)h->npts;
  PointTable t;
  t.x = base;
  t.y = base + np;
  t.nx = base + 2 * np;
  t.ny = base + 3 * np;
  t.w = base + 4 * np;
  t.kappa = base + 5 * np;
  t.hs = base + 6 * np;
  t.id = reinterpret_cast<const int*>(base + 7 * np);
  return t;
}

KernelParams kparams(const symhss_params& p) { return make_kernel_params(p); }

int proxy_count(const symhss_params& p, double radius) {
  const double kmax = std::max(p.k0, p.k1);
  const int need = (int)std::ceil((2.0 * kmax * radius + 32.0) / 8.0) * 8;
  return std::max(p.nproxy, need);
}

int tree_depth(int n, int leaf) {
  if (n <= leaf) return 0;
  return (int)std::ceil(std::log2((double)n / (double)leaf));
}

int read_status(symhss_s* h, cudaStream_t s) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st & ST_BAD_INDEX) return SYMHSS_ERR_DEVICE;
  if (st & ST_RANK_OVERFLOW) return SYMHSS_ERR_RANK_OVERFLOW;
  if (st & ST_SINGULAR) return SYMHSS_ERR_SINGULAR;
  if (st & ST_TIMEOUT) return SYMHSS_ERR_TIMEOUT;
  if (st) return SYMHSS_ERR_DEVICE;
  return SYMHSS_OK;
}

// The boxes of every problem at height t (level depth - t), problems in order;
// roots (height = depth) only if `with_roots`.
void height_boxes(symhss_s* h, int t, bool with_roots, std::vector<BoxRef>& out) {
  out.clear();
  for (int p = 0; p < (int)h->probs.size(); ++p) {
    Problem& P = h->probs[p];
    if (P.depth < t || (P.depth == t && !with_roots)) continue;
    const int l = P.depth - t;
    auto& bxs = P.levels[l];
    for (int b = 0; b < (int)bxs.size(); ++b) out.push_back(BoxRef{p, l, b, &bxs[b]});
  }
}

// Build the trees (host) and the point table (nodes of every problem, then the proxy rings).
int build_geometry(symhss_s* h, cudaStream_t s) {
  int node0 = 0;
  h->maxdepth = 0;
  h->max_n = 0;
  for (Problem& P : h->probs) {
    P.depth = tree_depth(P.n, P.prm.leaf);
    if (P.depth >= SYMHSS_MAX_LEVELS) return SYMHSS_ERR_INVALID;
    P.node0 = node0;
    P.vec0 = 2LL * node0;
    node0 += P.n;
    h->maxdepth = std::max(h->maxdepth, P.depth);
    h->max_n = std::max(h->max_n, P.n);
  }
  h->ntot = node0;
  // keep the heights' device buffers when the tallest tree is unchanged (set_curve)
  if ((int)h->heights.size() != h->maxdepth + 1) {
    h->heights.clear();
    h->heights.resize(h->maxdepth + 1);
  }
  for (Problem& P : h->probs) {
    P.levels.assign(P.depth + 1, {});
    P.levels[0].resize(1);
    P.levels[0][0].begin = P.node0;
    P.levels[0][0].end = P.node0 + P.n;
    for (int l = 1; l <= P.depth; ++l) {
      auto& prev = P.levels[l - 1];
      auto& cur = P.levels[l];
      cur.resize(2 * prev.size());
      for (size_t i = 0; i < prev.size(); ++i) {
        const int b = prev[i].begin, e = prev[i].end, mid = b + (e - b) / 2;
        cur[2 * i].begin = b; cur[2 * i].end = mid;
        cur[2 * i + 1].begin = mid; cur[2 * i + 1].end = e;
        prev[i].child[0] = (int)(2 * i);
        prev[i].child[1] = (int)(2 * i + 1);
      }
    }
  }
  int npts = h->ntot;
  for (Problem& P : h->probs) {
    for (int l = 0; l <= P.depth; ++l) {
      for (auto& bx : P.levels[l]) {
        const int cnt = bx.end - bx.begin;
        double sx = 0, sy = 0;
        for (int i = bx.begin; i < bx.end; ++i) { sx += h->hx[i]; sy += h->hy[i]; }
        bx.cx = cnt ? sx / cnt : 0.0;
        bx.cy = cnt ? sy / cnt : 0.0;
        double rho = 0;
        for (int i = bx.begin; i < bx.end; ++i) rho = std::max(rho, std::hypot(h->hx[i] - bx.cx, h->hy[i] - bx.cy));
        bx.rho = rho;
        bx.R = P.prm.proxy_factor * rho;
        if (l > 0) {
          bx.P = proxy_count(P.prm, bx.R);
          bx.proxy0 = npts;
          npts += bx.P;
        }
      }
    }
  }
  h->npts = npts;
  const size_t np = (size_t)npts;
  std::vector<double> tab(8 * np, 0.0);
  double *X = tab.data(), *Y = X + np, *NX = Y + np, *NY = NX + np, *W = NY + np, *K = W + np, *HS = K + np;
  int* ID = reinterpret_cast<int*>(HS + np);
  for (int i = 0; i < h->ntot; ++i) {
    X[i] = h->hx[i]; Y[i] = h->hy[i]; NX[i] = h->hnx[i]; NY[i] = h->hny[i]; W[i] = h->hw[i]; K[i] = h->hk[i];
    ID[i] = i;
  }
  // speed term of the hypersingular diagonal, per closed curve (problem); zero at proxies
  for (const Problem& P : h->probs) speed_terms(h->hw.data() + P.node0, P.n, HS + P.node0);
  for (Problem& P : h->probs) {
    for (int l = 1; l <= P.depth; ++l) {
      for (auto& bx : P.levels[l]) {
        for (int m = 0; m < bx.P; ++m) {
          const double phi = 2.0 * kPi * m / bx.P;
          const double c = std::cos(phi), sn = std::sin(phi);
          const int q = bx.proxy0 + m;
          X[q] = bx.cx + bx.R * c; Y[q] = bx.cy + bx.R * sn; NX[q] = c; NY[q] = sn;
          W[q] = 2.0 * kPi * bx.R / bx.P; K[q] = 0.0; ID[q] = -1;
        }
      }
    }
  }
  CK(h->pts.ensure(tab.size() * sizeof(double)));
  CK(cudaMemcpyAsync(h->pts.p, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  std::vector<KernelParams> kp;
  std::vector<WaveJob> wv;
  for (const Problem& P : h->probs) {
    kp.push_back(kparams(P.prm));
    WaveJob wj;
    wj.node0 = P.node0; wj.n = P.n; wj.vec0 = P.vec0; wj.k0 = P.prm.k0;
    const double2 z = make_double2(0.0, 0.0);
    if (P.prm.formulation == SYMHSS_BM) {  // [-u_in - (i/k0) du_in/dnu ; 0]
      wj.a1 = make_double2(-1.0, 0.0); wj.b1 = make_double2(0.0, -1.0 / P.prm.k0); wj.a2 = z; wj.b2 = z;
    } else if (P.prm.formulation == SYMHSS_PMCHWT) {  // [-u_in ; du_in/dnu / eps0]
      wj.a1 = make_double2(-1.0, 0.0); wj.b1 = z; wj.a2 = z; wj.b2 = make_double2(1.0 / P.prm.eps0, 0.0);
    } else {  // [-eps0 u_in ; du_in/dnu]
      wj.a1 = make_double2(-P.prm.eps0, 0.0); wj.b1 = z; wj.a2 = z; wj.b2 = make_double2(1.0, 0.0);
    }
    wv.push_back(wj);
  }
  CK(h->kps.ensure(kp.size() * sizeof(KernelParams)));
  CK(cudaMemcpyAsync(h->kps.p, kp.data(), kp.size() * sizeof(KernelParams), cudaMemcpyHostToDevice, s));
  CK(h->waves.ensure(wv.size() * sizeof(WaveJob)));
  CK(cudaMemcpyAsync(h->waves.p, wv.data(), wv.size() * sizeof(WaveJob), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // the host arrays are pageable and go out of scope
  h->mark.assign(np, -1);
  return SYMHSS_OK;
}

// Merge two ordered point lists carrying slots into "points with two slots".
// list0[i] gets slot base0 + i, list1[i] gets slot base1 + i.
void merge_slots(std::vector<int>& mark, const std::vector<int>& list0, int base0,
                 const std::vector<int>& list1, int base1, std::vector<int>& pt, std::vector<int>& s0,
                 std::vector<int>& s1) {
  for (size_t i = 0; i < list1.size(); ++i) mark[list1[i]] = base1 + (int)i;
  for (size_t i = 0; i < list0.size(); ++i) {
    const int q = list0[i];
    pt.push_back(q);
    s0.push_back(base0 + (int)i);
    s1.push_back(mark[q]);
    mark[q] = -2;
  }
  for (size_t i = 0; i < list1.size(); ++i) {
    const int q = list1[i];
    if (mark[q] >= 0) {
      pt.push_back(q);
      s0.push_back(-1);
      s1.push_back(mark[q]);
    }
  }
  for (int q : list1) mark[q] = -1;
  for (int q : list0) mark[q] = -1;
}

struct TileBuilder {
  std::vector<int> tp_pt, tp_s0, tp_s1, lp_pt, lp_s0, lp_s1;
  std::vector<TileJob> jobs;
  std::vector<TileChunk> chunks;
  long long pairs = 0;
  // thread points from (list0 -> slot base0+i, list1 -> base1+i); loop points likewise;
  // `prm`: the problem whose constants the tile uses
  void add(std::vector<int>& mark, const std::vector<int>& t0, int tb0, const std::vector<int>& t1, int tb1,
           const std::vector<int>& l0, int lb0, const std::vector<int>& l1, int lb1, long long out_off, int ld,
           int flags, int prm) {
    TileJob jb;
    jb.tp_off = (int)tp_pt.size();
    merge_slots(mark, t0, tb0, t1, tb1, tp_pt, tp_s0, tp_s1);
    jb.n_tp = (int)tp_pt.size() - jb.tp_off;
    jb.lp_off = (int)lp_pt.size();
    merge_slots(mark, l0, lb0, l1, lb1, lp_pt, lp_s0, lp_s1);
    jb.n_lp = (int)lp_pt.size() - jb.lp_off;
    jb.out_off = out_off;
    jb.ld = ld;
    jb.flags = flags;
    jb.prm = prm;
    jb.pad_ = 0;
    if (jb.n_tp == 0 || jb.n_lp == 0) return;
    jobs.push_back(jb);
    pairs += (flags & TILE_SYM_DIAG) ? (long long)jb.n_tp * (jb.n_tp + 1) / 2 : (long long)jb.n_tp * jb.n_lp;
  }
  // chunks of TILE_T thread points x ln loop points; a launch that would leave most SMs
  // idle uses shorter loop chunks (more blocks, each with less work)
  void make_chunks(int fixed_ln) {
    long long base = 0;
    for (const TileJob& jb : jobs)
      base += (long long)((jb.n_tp + TILE_T - 1) / TILE_T) * ((jb.n_lp + TILE_L - 1) / TILE_L);
    const int sms = device_sm_count();
    int ln = base >= 4 * sms ? TILE_L : (base >= 2 * sms ? TILE_L / 2 : TILE_L / 4);
    if (fixed_ln > 0) ln = std::min(fixed_ln, TILE_L);
    chunks.clear();
    for (int j = 0; j < (int)jobs.size(); ++j)
      for (int a = 0; a < jobs[j].n_tp; a += TILE_T)
        for (int b = 0; b < jobs[j].n_lp; b += ln) {
          // a symmetric diagonal block: no chunk whose loop points all precede its thread points
          if ((jobs[j].flags & TILE_SYM_DIAG) && b + ln <= a) continue;
          chunks.push_back(TileChunk{j, a, b, ln});
        }
  }
  cudaError_t launch(symhss_s* h, DevBuf& buf, double2* out, cudaStream_t s) {
    if (jobs.empty()) return cudaSuccess;
    make_chunks(h->tune.tile_loop_chunk);
    Packer pk;
    const size_t o1 = pk.add(tp_pt), o2 = pk.add(tp_s0), o3 = pk.add(tp_s1);
    const size_t o4 = pk.add(lp_pt), o5 = pk.add(lp_s0), o6 = pk.add(lp_s1);
    const size_t o7 = pk.add(jobs), o8 = pk.add(chunks);
    cudaError_t e = pk.upload(buf, s);
    if (e != cudaSuccess) return e;
    char* base = buf.as<char>();
    TileLaunch a;
    a.tpts = table_of(h);
    a.lpts = a.tpts;
    a.tp_pt = reinterpret_cast<const int*>(base + o1);
    a.tp_s0 = reinterpret_cast<const int*>(base + o2);
    a.tp_s1 = reinterpret_cast<const int*>(base + o3);
    a.lp_pt = reinterpret_cast<const int*>(base + o4);
    a.lp_s0 = reinterpret_cast<const int*>(base + o5);
    a.lp_s1 = reinterpret_cast<const int*>(base + o6);
    a.jobs = reinterpret_cast<const TileJob*>(base + o7);
    a.chunks = reinterpret_cast<const TileChunk*>(base + o8);
    a.nchunks = (int)chunks.size();
    a.out = out;
    a.status = h->status.as<int>();
    a.kps = h->kps.as<KernelParams>();
    return launch_tiles(a, s);
  }
};

inline long long tcap(int n) { return (long long)(n / 2) * ((n + 1) / 2) + 1; }

// Sketch rows held out of each sketched ID to estimate its residual on the proxy matrix.
constexpr int kHoldRows = 16;

// Near points of box b among the active lists of the other boxes of its level
// (row lists if `rows`, else column lists), part `part`.
void near_points(const symhss_s* h, const std::vector<HBox>& lev, int b, bool rows, int part,
                 std::vector<int>& out) {
  const HBox& bx = lev[b];
  out.clear();
  for (size_t o = 0; o < lev.size(); ++o) {
    if ((int)o == b) continue;
    const HBox& ot = lev[o];
    if (std::hypot(ot.cx - bx.cx, ot.cy - bx.cy) >= bx.R + ot.rho) continue;
    const std::vector<int>& ids = rows ? ot.actrow[part] : ot.act[part];
    for (int q : ids)
      if (std::hypot(h->hx[q] - bx.cx, h->hy[q] - bx.cy) < bx.R) out.push_back(q);
  }
}

// Fixed rank of Sec. 4.3 at height t (level L - t): ceil(a^t kL); -1 with tolerance ranks.
int fixed_rank(const symhss_s* h, int t) {
  if (h->prm.fixed_rank_kL <= 0) return -1;
  return (int)std::ceil(std::pow(h->prm.rank_scale_a, t) * h->prm.fixed_rank_kL);
}

int compress_height(symhss_s* h, int t, cudaStream_t s) {
  Height& H = h->heights[t];
  std::vector<BoxRef> refs;
  height_boxes(h, t, false, refs);
  const int nb = (int)refs.size();
  if (nb == 0) return SYMHSS_OK;
  const bool sym = h->prm.mode == SYMHSS_SYM;
  // active sets
  for (const BoxRef& rf : refs) {
    HBox& bx = *rf.bx;
    if (t == 0) {
      std::vector<int> ids(bx.end - bx.begin);
      for (int i = 0; i < (int)ids.size(); ++i) ids[i] = bx.begin + i;
      for (int p = 0; p < 2; ++p) { bx.act[p] = ids; bx.actrow[p] = ids; }
    } else {
      const auto& kids = h->probs[rf.p].levels[rf.l + 1];
      const HBox& c1 = kids[bx.child[0]];
      const HBox& c2 = kids[bx.child[1]];
      for (int p = 0; p < 2; ++p) {
        bx.act[p].assign(c1.perm[p].begin(), c1.perm[p].begin() + c1.rank[p]);
        for (int& v : bx.act[p]) v = c1.act[p][v];
        for (int j = 0; j < c2.rank[p]; ++j) bx.act[p].push_back(c2.act[p][c2.perm[p][j]]);
        bx.actrow[p].clear();
        for (int j = 0; j < c1.rrank[p]; ++j) bx.actrow[p].push_back(c1.actrow[p][c1.rperm[p][j]]);
        for (int j = 0; j < c2.rrank[p]; ++j) bx.actrow[p].push_back(c2.actrow[p][c2.rperm[p][j]]);
      }
    }
  }
  TileBuilder tb;
  std::vector<IdJob> jobs;
  long long mr_total = 0, t_total = 0, perm_total = 0;
  int max_m = 1, max_n = 1;
  const int fixed = fixed_rank(h, t);
  std::vector<int> nr0, nr1, prx0;
  const int flags = sym ? 0 : TILE_UNSCALED;
  // M_R of every box (and M_L^T for the baseline)
  for (int i = 0; i < nb; ++i) {
    const BoxRef& rf = refs[i];
    HBox& bx = *rf.bx;
    const auto& lev = h->probs[rf.p].levels[rf.l];
    near_points(h, lev, rf.b, true, 0, nr0);
    near_points(h, lev, rf.b, true, 1, nr1);
    prx0.resize(bx.P);
    for (int m = 0; m < bx.P; ++m) prx0[m] = bx.proxy0 + m;
    const int m0 = (int)nr0.size(), m1 = (int)nr1.size(), P = bx.P;
    const int m = m0 + m1 + 2 * P;
    const int n0 = (int)bx.act[0].size(), n1 = (int)bx.act[1].size();
    bx.m_near = m0 + m1;
    // rows: near eq1 (slots 0..m0), near eq2 (m0..), proxy eq1 and eq2 (same points)
    tb.add(h->mark, nr0, 0, nr1, m0, bx.act[0], 0, bx.act[1], n0, mr_total, m, flags, rf.p);
    tb.add(h->mark, prx0, m0 + m1, prx0, m0 + m1 + P, bx.act[0], 0, bx.act[1], n0, mr_total, m, flags, rf.p);
    for (int p = 0; p < 2; ++p) {
      IdJob j;
      j.m_off = mr_total + (p == 0 ? 0 : (long long)n0 * m);
      j.m = m; j.n = p == 0 ? n0 : n1; j.ld = m;
      j.start = 0; j.fixed = fixed;
      j.t_off = t_total; t_total += tcap(j.n);
      j.perm_off = perm_total; perm_total += j.n;
      j.out_idx = 2 * i + p;
      jobs.push_back(j);
      bx.t_off[p] = j.t_off;
      max_n = std::max(max_n, j.n);
    }
    max_m = std::max(max_m, m);
    mr_total += (long long)m * (n0 + n1);
  }
  if (!sym) {
    for (int i = 0; i < nb; ++i) {
      const BoxRef& rf = refs[i];
      HBox& bx = *rf.bx;
      const auto& lev = h->probs[rf.p].levels[rf.l];
      near_points(h, lev, rf.b, false, 0, nr0);
      near_points(h, lev, rf.b, false, 1, nr1);
      prx0.resize(bx.P);
      for (int m = 0; m < bx.P; ++m) prx0[m] = bx.proxy0 + m;
      const int c0 = (int)nr0.size(), c1n = (int)nr1.size(), P = bx.P;
      const int mt = c0 + c1n + 2 * P;  // rows of M_L^T = columns of M_L
      const int r0 = (int)bx.actrow[0].size(), r1 = (int)bx.actrow[1].size();
      // thread points = M_L columns (sources), loop points = M_L rows (observations)
      tb.add(h->mark, nr0, 0, nr1, c0, bx.actrow[0], 0, bx.actrow[1], r0, mr_total, mt,
             flags | TILE_SRC_IS_THREAD, rf.p);
      tb.add(h->mark, prx0, c0 + c1n, prx0, c0 + c1n + P, bx.actrow[0], 0, bx.actrow[1], r0, mr_total, mt,
             flags | TILE_SRC_IS_THREAD, rf.p);
      for (int p = 0; p < 2; ++p) {
        IdJob j;
        j.m_off = mr_total + (p == 0 ? 0 : (long long)r0 * mt);
        j.m = mt; j.n = p == 0 ? r0 : r1; j.ld = mt;
        j.start = 0; j.fixed = fixed;
        j.t_off = t_total; t_total += tcap(j.n);
        j.perm_off = perm_total; perm_total += j.n;
        j.out_idx = 2 * nb + 2 * i + p;
        jobs.push_back(j);
        bx.rt_off[p] = j.t_off;
        max_n = std::max(max_n, j.n);
      }
      max_m = std::max(max_m, mt);
      mr_total += (long long)mt * (r0 + r1);
    }
  }
  const int njobs = (int)jobs.size();
  const int p_over = h->prm.oversample;
  // Proposed ranks of the attached network (features and forward pass on the device),
  // read back before the tiles are launched so that the host can size the sketches
  // while the tiles run.
  std::vector<float> prop;  // nb x 2 outputs
  if (h->mlp && p_over > 0 && fixed < 0) {
    std::vector<FeatJob> fj(nb);
    for (int i = 0; i < nb; ++i) {
      const BoxRef& rf = refs[i];
      const HBox& bx = *rf.bx;
      const symhss_params& pp = h->probs[rf.p].prm;
      FeatJob f;
      f.cx = bx.cx; f.cy = bx.cy; f.rho = bx.rho; f.k0 = pp.k0; f.k1 = pp.k1; f.tol = h->prm.tol;
      f.begin = bx.begin; f.len = bx.end - bx.begin; f.height = t;
      f.n0 = (int)bx.act[0].size(); f.n1 = (int)bx.act[1].size(); f.m_near = bx.m_near; f.nproxy = bx.P;
      f.pad_ = 0;
      fj[i] = f;
    }
    Packer fp;
    fp.add(fj);
    CK(fp.upload(h->featjobs, s));
    CK(h->feats.ensure((size_t)nb * kMlpWidth * sizeof(float)));
    CK(h->mlpout.ensure((size_t)nb * kMlpWidth * sizeof(float)));
    const int e0 = prof_begin(h, s);
    CK(launch_box_features(table_of(h), h->featjobs.as<FeatJob>(), nb, h->feats.as<float>(), s));
    CK(mlp_forward(h->mlp, h->feats.as<float>(), nb, h->mlpout.as<float>(), s));
    prof_end(h, s, SYMHSS_K_MLP, e0, 2.0 * 3 * kMlpWidth * kMlpWidth * (double)nb);
    prop.resize((size_t)nb * 2);
    CK(cudaMemcpy2DAsync(prop.data(), 2 * sizeof(float), h->mlpout.p, kMlpWidth * sizeof(float),
                         2 * sizeof(float), nb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  // Randomized sketch (Halko-Martinsson-Tropp): an ID job whose rank estimate plus
  // oversampling is well below its row count is taken of Y = Omega M instead of M.
  // Y blocks live after all proxy matrices in the same buffer.  Rank estimate: the
  // network's proposal times the margin when a network is attached; else, at the leaves,
  // 3 log10(1/tol) + 2 k rho + 12 (at most half the smaller dimension), and above, 1.7x the
  // problem's largest rank one level down.
  const std::vector<IdJob> full = jobs;  // the same IDs on the full proxy matrices
  std::vector<int> sk_rows(njobs, 0);
  std::vector<SketchJob> sk;
  std::vector<SketchColWork> skcw;
  std::vector<SketchTile> sktiles;
  long long y_total = 0, slice_total = 0, exp_total = 0;
  double sketch_work = 0;
  if (p_over > 0) {
    for (int i = 0; i < njobs; ++i) {
      IdJob& j = jobs[i];
      if (j.n == 0) continue;
      const int part = j.out_idx & 1;
      const int bi = (j.out_idx % (2 * nb)) / 2;
      const BoxRef& rf = refs[bi];
      int est;
      if (fixed >= 0) est = fixed;
      else if (!prop.empty()) {
        const double r = std::exp2(8.0 * (double)prop[2 * bi + part]) - 1.0;
        est = (int)std::ceil(h->prop_margin * std::max(0.0, std::min(r, 1e6))) + 2;
      } else if (t == 0) {
        // leaves: a box of radius rho sees about 2 k rho oscillations plus a few terms per
        // decade of the tolerance (the proxy expansion's length); never above half the smaller
        // dimension.  The held-out check and the redo path still decide every ID.
        const symhss_params& pp = h->probs[rf.p].prm;
        const double kr = std::max(pp.k0, pp.k1) * rf.bx->rho;
        const double dec = std::log10(1.0 / std::max(1e-300, h->prm.tol));
        est = std::min((std::min(j.m, j.n) + 1) / 2, (int)std::ceil(3.0 * dec + 2.0 * kr) + 12);
      } else est = (int)std::ceil(1.7 * std::max(8, h->probs[rf.p].lvl_max_rank[rf.l + 1][part]));
      const int sr = std::max(32, ((est + p_over + 15) / 16) * 16);
      const int stot = sr + kHoldRows;  // rows for the ID, then held-out rows for its check
      if (stot > 1024 || 5 * stot >= 4 * j.m) continue;
      SketchJob sj;
      sj.m_off = j.m_off; sj.m = j.m; sj.n = j.n; sj.ld = j.ld;
      sj.mpad = sketch_mpad(j.m); sj.n2pad = sketch_n2pad(j.n); sj.s = stot;
      sj.y_off = mr_total + y_total; sj.ldy = stot;
      sj.slice_off = slice_total; sj.exp_off = exp_total;
      sj.stream_id = ((long long)t << 32) + i;
      const int sji = (int)sk.size();
      for (int c = 0; c < j.n; ++c) skcw.push_back(SketchColWork{sji, c});
      const int mtiles = (stot + 127) / 128;
      for (int cb = 0; cb < sj.n2pad / 32; ++cb)
        for (int mt = 0; mt < mtiles; ++mt) sktiles.push_back(SketchTile{sji, cb, mt});
      // algorithmic work of Y = Omega M: an s x m by m x n complex product, 8 s m n real flops
      sketch_work += 8.0 * (double)stot * (double)j.m * (double)j.n;
      y_total += (long long)stot * j.n;
      slice_total += (long long)sketch_slice_bytes(sj.mpad, sj.n2pad);
      exp_total += 2LL * j.n;
      sk.push_back(sj);
      sk_rows[i] = sr;
      j.m_off = sj.y_off; j.m = sr; j.ld = stot;
    }
  }
  max_m = 1;
  for (const IdJob& j : jobs) max_m = std::max(max_m, j.m);
  CK(H.mr.ensure((mr_total + y_total) * sizeof(double2)));
  CK(H.tbuf.ensure(t_total * sizeof(double2)));
  CK(H.permbuf.ensure(perm_total * sizeof(int)));
  CK(H.rankbuf.ensure(njobs * sizeof(int)));
  CK(H.refbuf.ensure(njobs * sizeof(double)));
  TIMED(SYMHSS_K_TILES, (double)tb.pairs, tb.launch(h, H.clists, H.mr.as<double2>(), s));
  if (!sk.empty()) {
    CK(H.slices.ensure((size_t)slice_total));
    Packer sp;
    const size_t oj = sp.add(sk), oc = sp.add(skcw), ot = sp.add(sktiles);
    const size_t oe = sp.add(nullptr, (size_t)exp_total * sizeof(int));
    CK(sp.upload(H.skmeta, s));
    char* sb = H.skmeta.as<char>();
    SketchLaunch sa;
    sa.mats = H.mr.as<double2>();
    sa.slices = H.slices.as<uint8_t>();
    sa.exps = reinterpret_cast<int*>(sb + oe);
    sa.y = H.mr.as<double2>();
    sa.jobs = reinterpret_cast<const SketchJob*>(sb + oj);
    sa.colwork = reinterpret_cast<const SketchColWork*>(sb + oc);
    sa.ncolwork = (int)skcw.size();
    sa.tiles = reinterpret_cast<const SketchTile*>(sb + ot);
    sa.ntiles = (int)sktiles.size();
    sa.seed = h->prm.seed;
    sa.status = h->status.as<int>();
    TIMED(SYMHSS_K_SKETCH, sketch_work, launch_sketch(sa, s));
  }
  // IDs of sketches use tol / 4: the sketch compresses the trailing pivot ratios, and at
  // tol / 4 the interpolation residual on M stays at or below that of the plain ID
  std::vector<IdJob> plain_jobs, sketch_jobs;
  for (int i = 0; i < njobs; ++i) (sk_rows[i] > 0 ? sketch_jobs : plain_jobs).push_back(jobs[i]);
  Packer pk;
  const size_t o_plain = pk.add(plain_jobs), o_sketch = pk.add(sketch_jobs);
  CK(pk.upload(H.idjobs, s));
  IdLaunch ia;
  ia.mats = H.mr.as<double2>();
  ia.tbuf = H.tbuf.as<double2>();
  ia.perm = H.permbuf.as<int>();
  ia.rank = H.rankbuf.as<int>();
  ia.ref = H.refbuf.as<double>();
  ia.tol = h->prm.tol;
  ia.status = h->status.as<int>();
  ia.max_m = max_m;
  ia.max_n = max_n;
  ia.cluster_max = h->tune.id_cluster_max;
  const size_t id_before = h->marks.size();
  ia.jobs = reinterpret_cast<const IdJob*>(H.idjobs.as<char>() + o_plain);
  ia.njobs = (int)plain_jobs.size();
  TIMED(SYMHSS_K_ID, 0.0, launch_cpqr(ia, s));
  ia.jobs = reinterpret_cast<const IdJob*>(H.idjobs.as<char>() + o_sketch);
  ia.njobs = (int)sketch_jobs.size();
  ia.tol = 0.25 * h->prm.tol;
  TIMED(SYMHSS_K_ID, 0.0, launch_cpqr(ia, s));
  ia.tol = h->prm.tol;
  const size_t id_mark = h->marks.size() > id_before ? id_before : (size_t)-1;
  // residual check of every sketched ID.  Without a proposer: its interpolation of the
  // held-out sketch rows Omega_h M (Halko-Martinsson-Tropp, Sec. 4.3 of their survey:
  // ||Omega_h e|| / sqrt(q) estimates ||e|| for Rademacher Omega_h with q rows).  With a
  // proposer attached, the ID of a proposed sketch is accepted on its residual on the proxy
  // matrix itself, max_c ||m_c - M_J t_c|| <= tol max_c ||m_c|| (the bound a plain ID meets by
  // construction: its stopping pivot is the largest remaining column norm).
  const bool proxy_check = h->mlp != nullptr;
  auto check_rows = [&](int i) {
    CheckJob c;
    if (proxy_check) {
      c.m_off = full[i].m_off; c.m = full[i].m; c.n = full[i].n; c.ld = full[i].ld;
    } else {
      c.m_off = jobs[i].m_off + sk_rows[i]; c.m = kHoldRows; c.n = jobs[i].n; c.ld = jobs[i].ld;
    }
    return c;
  };
  std::vector<int> chk_of(njobs, -1);
  std::vector<double> ratio;
  if (!sketch_jobs.empty() && !proxy_check) {
    std::vector<CheckJob> cj;
    for (int i = 0; i < njobs; ++i) {
      if (sk_rows[i] == 0) continue;
      CheckJob c = check_rows(i);
      c.rank_idx = jobs[i].out_idx; c.t_off = jobs[i].t_off; c.perm_off = jobs[i].perm_off;
      c.out = (int)cj.size(); c.pad_ = 0;
      chk_of[i] = c.out;
      cj.push_back(c);
    }
    Packer cp;
    cp.add(cj);
    CK(cp.upload(h->chkjobs, s));
    CK(h->chkratio.ensure(cj.size() * 3 * sizeof(double)));  // ratios, then the check's maxima
    TIMED(SYMHSS_K_CHECK, 0.0, launch_id_check(H.mr.as<double2>(), H.tbuf.as<double2>(), H.permbuf.as<int>(),
                                               H.rankbuf.as<int>(), h->chkjobs.as<CheckJob>(), (int)cj.size(),
                                               h->chkratio.as<double>(), s));
    ratio.resize(cj.size());
    CK(cudaMemcpyAsync(ratio.data(), h->chkratio.p, cj.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  std::vector<int> hr(njobs), hp(perm_total);
  CK(cudaMemcpyAsync(hr.data(), H.rankbuf.p, njobs * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hp.data(), H.permbuf.p, perm_total * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // exact residual of the given sketched IDs on their proxy matrices (ranks and permutations
  // read back above): gather M_J and M_rest, M_rest -= M_J T on the tensor cores, ratio of the
  // largest residual column norm to the largest column norm of M
  auto proxy_ratios = [&](const std::vector<int>& ids, std::vector<double>& out) -> int {
    out.assign(ids.size(), 0.0);
    if (ids.empty()) return SYMHSS_OK;
    std::vector<GatherJob> gj;
    std::vector<int2> work;
    std::vector<int> outs;
    long long gtot = 0;
    int maxr = 0;
    for (size_t k = 0; k < ids.size(); ++k) {
      const int i = ids[k];
      GatherJob g;
      g.m_off = full[i].m_off; g.m = full[i].m; g.n = full[i].n; g.ld = full[i].ld;
      g.r = std::min(std::max(hr[jobs[i].out_idx], 0), g.n);
      g.perm_off = jobs[i].perm_off;
      g.g1_off = gtot;
      g.g2_off = gtot + (long long)g.m * g.r;
      gtot += (long long)g.m * g.n;
      maxr = std::max(maxr, g.r);
      for (int c = 0; c < g.n; ++c) work.push_back(make_int2((int)gj.size(), c));
      outs.push_back((int)k);
      gj.push_back(g);
    }
    const int TM = zgemm_tc_tile_rows(), TN = zgemm_tc_tile_cols(), KM = zgemm_tc_max_k();
    const int nchunk = (maxr + KM - 1) / KM;
    std::vector<std::vector<ZgemmJob>> zj(nchunk);
    std::vector<std::vector<ZgemmTile>> zt(nchunk);
    int zmt = 1, znt = 1;  // the largest row / column block counts of the products
    for (size_t k = 0; k < ids.size(); ++k) {
      const GatherJob& g = gj[k];
      const int rest = g.n - g.r;
      if (g.r == 0 || rest == 0) continue;
      for (int c = 0; c * KM < g.r; ++c) {
        ZgemmJob z;
        z.a_off = g.g1_off + (long long)c * KM * g.m; z.lda = g.m;
        z.b_off = jobs[ids[k]].t_off + (long long)c * KM; z.ldb = g.r;
        z.c_off = g.g2_off; z.ldc = g.m;
        z.m = g.m; z.n = rest; z.k = std::min(KM, g.r - c * KM);
        const int jid = (int)zj[c].size();
        zj[c].push_back(z);
        zmt = std::max(zmt, (g.m + TM - 1) / TM);
        znt = std::max(znt, (rest + TN - 1) / TN);
        for (int a = 0; a < (g.m + TM - 1) / TM; ++a)
          for (int b = 0; b < (rest + TN - 1) / TN; ++b) zt[c].push_back(ZgemmTile{jid, a, b});
      }
    }
    Packer pg;
    const size_t og = pg.add(gj), ow = pg.add(work), oo = pg.add(outs);
    std::vector<size_t> ozj(nchunk), ozt(nchunk);
    for (int c = 0; c < nchunk; ++c) { ozj[c] = pg.add(zj[c]); ozt[c] = pg.add(zt[c]); }
    CK(pg.upload(H.chkmeta, s));
    CK(H.chkg.ensure((size_t)gtot * sizeof(double2)));
    size_t zmax = 0;
    for (int c = 0; c < nchunk; ++c) zmax = std::max(zmax, zj[c].size());
    CK(H.chkimg.ensure((size_t)zgemm_img_bytes((int)zmax, zmt, znt)));
    CK(h->chkratio.ensure(ids.size() * sizeof(double)));
    const char* mb = H.chkmeta.as<char>();
    double w = 0;
    for (const GatherJob& g : gj) w += 8.0 * (double)g.m * g.r * (g.n - g.r);
    const int e0 = prof_begin(h, s);
    CK(launch_gather_cols(H.mr.as<double2>(), H.permbuf.as<int>(), reinterpret_cast<const GatherJob*>(mb + og),
                          reinterpret_cast<const int2*>(mb + ow), (int)work.size(), H.chkg.as<double2>(), s));
    for (int c = 0; c < nchunk; ++c) {
      if (zt[c].empty()) continue;
      ZgemmLaunch za;
      za.A = H.chkg.as<double2>(); za.B = H.tbuf.as<double2>(); za.C = H.chkg.as<double2>();
      za.jobs = reinterpret_cast<const ZgemmJob*>(mb + ozj[c]);
      za.tiles = reinterpret_cast<const ZgemmTile*>(mb + ozt[c]);
      za.ntiles = (int)zt[c].size();
      za.mode = ZGEMM_SUB;
      za.status = h->status.as<int>();
      za.wait_ns = 0;
      za.njobs = (int)zj[c].size();
      za.mtiles = zmt;
      za.ntiles_c = znt;
      za.img = H.chkimg.as<unsigned char>();
      za.img_bytes = (long long)H.chkimg.cap;
      CK(launch_zgemm_tc(za, s));
    }
    CK(launch_residual_ratio(H.mr.as<double2>(), H.chkg.as<double2>(), reinterpret_cast<const GatherJob*>(mb + og),
                             reinterpret_cast<const int*>(mb + oo), (int)gj.size(), h->chkratio.as<double>(), s));
    prof_end(h, s, SYMHSS_K_CHECK, e0, w);
    CK(cudaMemcpyAsync(out.data(), h->chkratio.p, ids.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return read_status(h, s);
  };
  if (!sketch_jobs.empty() && proxy_check) {
    std::vector<int> ids;
    for (int i = 0; i < njobs; ++i)
      if (sk_rows[i] != 0) { chk_of[i] = (int)ids.size(); ids.push_back(i); }
    const int rc = proxy_ratios(ids, ratio);
    if (rc) return rc;
  }
  if (!prop.empty()) {
    for (int i = 0; i < njobs; ++i) {
      if (jobs[i].n == 0 || jobs[i].out_idx >= 2 * nb) continue;
      const int bi = jobs[i].out_idx / 2, part = jobs[i].out_idx & 1;
      const double r = std::exp2(8.0 * (double)prop[2 * bi + part]) - 1.0;
      const int ri = hr[jobs[i].out_idx];
      h->st.proposals += 1;
      h->st.proposal_rank_err += std::fabs(r - ri) / std::max(1, ri);
      if (r < ri) h->st.proposal_under += 1;
    }
  }
  if (id_mark < h->marks.size()) {
    double w = 0;
    for (const IdJob& j : jobs) w += id_flops(j.m, j.n, hr[j.out_idx]);
    h->marks[id_mark].work = w;
  }
  // A sketch too thin for the rank it revealed: redo that ID on the full matrix.  An ID
  // whose held-out residual exceeds tol: continue its pivoted QR on the sketch at tol / 16
  // (a few more skeleton columns) and check again; redo it on the full matrix only if it
  // still fails.
  std::vector<IdJob> cur = jobs;
  {
    std::vector<IdJob> redo;
    std::vector<int> cont;
    auto thin = [&](int i) { return fixed < 0 && 2 * hr[i] >= 2 * sk_rows[i] - p_over; };
    for (int i = 0; i < njobs; ++i) {
      if (sk_rows[i] == 0) continue;
      const double rt = chk_of[i] >= 0 ? ratio[chk_of[i]] : 0.0;
      if (thin(i)) {
        redo.push_back(full[i]);
        cur[i] = full[i];
      } else if (!(rt <= h->prm.tol)) {
        h->st.check_failed += 1;
        cont.push_back(i);
      } else {
        h->st.check_max_ratio = std::max(h->st.check_max_ratio, rt);
      }
    }
    if (!cont.empty()) {
      std::vector<IdJob> cjobs;
      std::vector<CheckJob> chk;
      int mm = 1;
      for (int i : cont) {
        IdJob j = jobs[i];
        j.start = hr[i];
        cjobs.push_back(j);
        mm = std::max(mm, j.m);
        CheckJob c = check_rows(i);
        c.rank_idx = jobs[i].out_idx; c.t_off = jobs[i].t_off; c.perm_off = jobs[i].perm_off;
        c.out = (int)chk.size(); c.pad_ = 0;
        chk.push_back(c);
      }
      Packer pc;
      const size_t oj = pc.add(cjobs), oc = pc.add(chk);
      CK(pc.upload(H.idjobs, s));
      ia.jobs = reinterpret_cast<const IdJob*>(H.idjobs.as<char>() + oj);
      ia.njobs = (int)cjobs.size();
      ia.max_m = mm;
      ia.tol = h->prm.tol / 16.0;
      const size_t cb = h->marks.size();
      TIMED(SYMHSS_K_ID, 0.0, launch_cpqr(ia, s));
      ia.tol = h->prm.tol;
      ia.max_m = max_m;
      std::vector<double> r2(chk.size());
      if (!proxy_check) {
        CK(h->chkratio.ensure(chk.size() * 3 * sizeof(double)));  // ratios, then the check's maxima
        TIMED(SYMHSS_K_CHECK, 0.0, launch_id_check(H.mr.as<double2>(), H.tbuf.as<double2>(), H.permbuf.as<int>(),
                                                   H.rankbuf.as<int>(),
                                                   reinterpret_cast<const CheckJob*>(H.idjobs.as<char>() + oc),
                                                   (int)chk.size(), h->chkratio.as<double>(), s));
        CK(cudaMemcpyAsync(r2.data(), h->chkratio.p, chk.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      }
      std::vector<int> before(cont.size());
      for (size_t k = 0; k < cont.size(); ++k) before[k] = hr[cont[k]];
      CK(cudaMemcpyAsync(hr.data(), H.rankbuf.p, njobs * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hp.data(), H.permbuf.p, perm_total * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (proxy_check) {
        const int rc = proxy_ratios(cont, r2);
        if (rc) return rc;
      }
      if (h->marks.size() > cb) {
        double w = 0;
        for (size_t k = 0; k < cont.size(); ++k) {
          const IdJob& j = jobs[cont[k]];
          w += id_flops(j.m, j.n, hr[j.out_idx]) - id_flops(j.m, j.n, before[k]);
        }
        h->marks[cb].work = w;
      }
      for (size_t k = 0; k < cont.size(); ++k) {
        const int i = cont[k];
        if (thin(i) || !(r2[k] <= h->prm.tol)) {
          redo.push_back(full[i]);
          cur[i] = full[i];
        } else {
          h->st.check_max_ratio = std::max(h->st.check_max_ratio, r2[k]);
        }
      }
    }
    h->st.sketch_redo += (long long)redo.size();
    if (!redo.empty()) {
      int mm = 1;
      for (const IdJob& j : redo) mm = std::max(mm, j.m);
      Packer pr;
      pr.add(redo);
      CK(pr.upload(H.idjobs, s));
      ia.jobs = H.idjobs.as<IdJob>();
      ia.njobs = (int)redo.size();
      ia.max_m = mm;
      const size_t rb = h->marks.size();
      TIMED(SYMHSS_K_ID, 0.0, launch_cpqr(ia, s));
      CK(cudaMemcpyAsync(hr.data(), H.rankbuf.p, njobs * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hp.data(), H.permbuf.p, perm_total * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (h->marks.size() > rb) {
        double w = 0;
        for (const IdJob& j : redo) w += id_flops(j.m, j.n, hr[j.out_idx]);
        h->marks[rb].work = w;
      }
      ia.max_m = max_m;
    }
  }
  h->st.pairs_evaluated += tb.pairs;
  if (!sym) {  // raise the lower of the row / column ranks of each half to the higher
    std::vector<IdJob> more;
    for (int b = 0; b < nb; ++b)
      for (int p = 0; p < 2; ++p) {
        const int ic = 2 * b + p, ir = 2 * nb + 2 * b + p;
        const int k = std::max(hr[ic], hr[ir]);
        for (int idx : {ic, ir}) {
          if (hr[idx] < k) {
            IdJob j = cur[idx];
            if (j.m_off != full[idx].m_off && 2 * k >= 2 * sk_rows[idx] - p_over) {
              j = full[idx];  // restart on the full matrix with the raised rank
              j.start = 0;
            } else {
              j.start = hr[idx];
            }
            j.fixed = k;
            more.push_back(j);
          }
        }
      }
    if (!more.empty()) {
      Packer pk2;
      pk2.add(more);
      CK(pk2.upload(H.idjobs, s));
      ia.jobs = H.idjobs.as<IdJob>();
      ia.njobs = (int)more.size();
      {
        int mm = 1;
        for (const IdJob& j : more) mm = std::max(mm, j.m);
        ia.max_m = mm;
      }
      const size_t more_before = h->marks.size();
      TIMED(SYMHSS_K_ID, 0.0, launch_cpqr(ia, s));
      const size_t more_mark = h->marks.size() > more_before ? more_before : (size_t)-1;
      CK(cudaMemcpyAsync(hr.data(), H.rankbuf.p, njobs * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hp.data(), H.permbuf.p, perm_total * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (more_mark < h->marks.size()) {
        double w = 0;
        for (const IdJob& j : more) w += id_flops(j.m, j.n, hr[j.out_idx]) - id_flops(j.m, j.n, j.start);
        h->marks[more_mark].work = w;
      }
    }
  }
  prof_collect(h);
  for (const IdJob& j : jobs) {
    const int r = hr[j.out_idx];
    h->st.flops_id += 16.0 * (double)j.m * j.n * r;
  }
  h->st.id_count += njobs;
  for (int i = 0; i < nb; ++i) {
    HBox& bx = *refs[i].bx;
    for (int p = 0; p < 2; ++p) {
      const IdJob& j = jobs[2 * i + p];
      bx.rank[p] = hr[2 * i + p];
      if (h->rank_limit > 0 && bx.rank[p] > h->rank_limit) return SYMHSS_ERR_RANK_OVERFLOW;
      bx.perm[p].assign(hp.begin() + j.perm_off, hp.begin() + j.perm_off + j.n);
      if (sym) {
        bx.rrank[p] = bx.rank[p];
        bx.rperm[p] = bx.perm[p];
        bx.rt_off[p] = bx.t_off[p];
      } else {
        const IdJob& jr = jobs[2 * nb + 2 * i + p];
        bx.rrank[p] = hr[jr.out_idx];
        if (h->rank_limit > 0 && bx.rrank[p] > h->rank_limit) return SYMHSS_ERR_RANK_OVERFLOW;
        bx.rperm[p].assign(hp.begin() + jr.perm_off, hp.begin() + jr.perm_off + jr.n);
        if (bx.rrank[p] != bx.rank[p]) return SYMHSS_ERR_DEVICE;
      }
    }
  }
  H.h_rank = hr;
  for (Problem& P : h->probs)
    if (P.depth > t) P.lvl_max_rank[P.depth - t][0] = P.lvl_max_rank[P.depth - t][1] = 0;
  for (const BoxRef& rf : refs)
    for (int p = 0; p < 2; ++p) {
      int& mx = h->probs[rf.p].lvl_max_rank[rf.l][p];
      mx = std::max(mx, rf.bx->rank[p]);
    }
  return SYMHSS_OK;
}

// Positions of each active unknown (part p, active order) in the box's diagonal-block
// ordering: leaf [flux; trace]; parent [child 1 (flux; trace), child 2 (flux; trace)].
void positions(const symhss_s* h, int t, const BoxRef& rf, bool rows, std::vector<int> pos[2]) {
  const HBox& bx = *rf.bx;
  if (t == 0) {
    const int nb = bx.end - bx.begin;
    for (int p = 0; p < 2; ++p) {
      pos[p].resize(nb);
      for (int i = 0; i < nb; ++i) pos[p][i] = p * nb + i;
    }
    return;
  }
  const auto& kids = h->probs[rf.p].levels[rf.l + 1];
  const HBox& c1 = kids[bx.child[0]];
  const HBox& c2 = kids[bx.child[1]];
  const int* r1 = rows ? c1.rrank : c1.rank;
  const int* r2 = rows ? c2.rrank : c2.rank;
  const int a1 = r1[0] + r1[1];
  for (int p = 0; p < 2; ++p) {
    pos[p].clear();
    const int o1 = p == 0 ? 0 : r1[0];
    const int o2 = a1 + (p == 0 ? 0 : r2[0]);
    for (int i = 0; i < r1[p]; ++i) pos[p].push_back(o1 + i);
    for (int i = 0; i < r2[p]; ++i) pos[p].push_back(o2 + i);
  }
}

// skeleton rows / columns of a box, per part, in pivot order
void skeleton(const HBox& bx, bool rows, int p, std::vector<int>& out) {
  out.clear();
  const std::vector<int>& a = rows ? bx.actrow[p] : bx.act[p];
  const std::vector<int>& pm = rows ? bx.rperm[p] : bx.perm[p];
  const int r = rows ? bx.rrank[p] : bx.rank[p];
  for (int j = 0; j < r; ++j) out.push_back(a[pm[j]]);
}

// Assemble the diagonal blocks D of every box at height t (leaf tiles, or children's
// Atilde plus skeleton coupling tiles) into H.D and factorise them (roots included).
int assemble_and_lu(symhss_s* h, int t, cudaStream_t s, long long& pairs) {
  Height& H = h->heights[t];
  std::vector<BoxRef> refs;
  height_boxes(h, t, true, refs);
  if (refs.empty()) return SYMHSS_OK;
  const bool sym = h->prm.mode == SYMHSS_SYM;
  const int flags = sym ? 0 : TILE_UNSCALED;
  const bool leaf = (t == 0);
  long long d_total = 0, piv_total = 0;
  int max_n = 1;
  for (const BoxRef& rf : refs) {
    HBox& bx = *rf.bx;
    if (leaf) bx.size = 2 * (bx.end - bx.begin);
    else {
      const auto& kids = h->probs[rf.p].levels[rf.l + 1];
      const HBox& c1 = kids[bx.child[0]];
      const HBox& c2 = kids[bx.child[1]];
      bx.size = c1.rank[0] + c1.rank[1] + c2.rank[0] + c2.rank[1];
    }
    bx.d_off = d_total;
    d_total += (long long)bx.size * bx.size;
    bx.piv_off = piv_total;
    piv_total += bx.size;
    max_n = std::max(max_n, bx.size);
  }
  CK(H.D.ensure(d_total * sizeof(double2)));
  CK(H.piv.ensure(piv_total * sizeof(int)));
  CK(H.perm.ensure(piv_total * sizeof(int)));
  CK(H.info.ensure(refs.size() * sizeof(int)));
  TileBuilder tb;
  std::vector<CopyJob> copies, mirrors;
  std::vector<int> t0, t1, u0, u1;
  for (const BoxRef& rf : refs) {
    HBox& bx = *rf.bx;
    if (leaf) {
      std::vector<int> ids(bx.end - bx.begin);
      for (int i = 0; i < (int)ids.size(); ++i) ids[i] = bx.begin + i;
      const int nb = (int)ids.size();
      // the leaf block is symmetric off its node diagonal in the symmetric system: one triangle
      tb.add(h->mark, ids, 0, ids, nb, ids, 0, ids, nb, bx.d_off, bx.size, sym ? flags | TILE_SYM_DIAG : flags, rf.p);
    } else {
      const auto& kids = h->probs[rf.p].levels[rf.l + 1];
      const HBox& c1 = kids[bx.child[0]];
      const HBox& c2 = kids[bx.child[1]];
      const int a1 = c1.rank[0] + c1.rank[1];
      // rows of child 1 against columns of child 2, and the transpose position
      skeleton(c1, true, 0, t0); skeleton(c1, true, 1, t1);
      skeleton(c2, false, 0, u0); skeleton(c2, false, 1, u1);
      tb.add(h->mark, t0, 0, t1, c1.rrank[0], u0, a1, u1, a1 + c2.rank[0], bx.d_off, bx.size, flags, rf.p);
      if (sym) {
        // one ID is both bases and the off-diagonal entries are symmetric, so the block of
        // child 2's rows against child 1's columns is the transpose of the one just tiled
        CopyJob tj;
        tj.src_off = bx.d_off + (long long)a1 * bx.size;
        tj.dst_off = bx.d_off + a1;
        tj.rows = a1;
        tj.cols = bx.size - a1;
        tj.lds = bx.size;
        tj.ldd = bx.size;
        tj.trans = 1;
        mirrors.push_back(tj);
      } else {
        skeleton(c2, true, 0, t0); skeleton(c2, true, 1, t1);
        skeleton(c1, false, 0, u0); skeleton(c1, false, 1, u1);
        tb.add(h->mark, t0, a1, t1, a1 + c2.rrank[0], u0, 0, u1, c1.rank[0], bx.d_off, bx.size, flags, rf.p);
      }
      CopyJob cj;
      cj.src_off = c1.rx_off; cj.dst_off = bx.d_off; cj.rows = a1; cj.cols = a1; cj.lds = a1; cj.ldd = bx.size;
      copies.push_back(cj);
      const int a2 = c2.rank[0] + c2.rank[1];
      cj.src_off = c2.rx_off; cj.dst_off = bx.d_off + a1 + (long long)a1 * bx.size;
      cj.rows = a2; cj.cols = a2; cj.lds = a2;
      copies.push_back(cj);
    }
  }
  TIMED(SYMHSS_K_TILES, (double)tb.pairs, tb.launch(h, H.flists, H.D.as<double2>(), s));
  pairs += tb.pairs;
  if (!copies.empty()) {
    Packer pk;
    pk.add(copies);
    const size_t om = pk.add(mirrors);
    CK(pk.upload(H.cjobs, s));
    if (!mirrors.empty())
      TIMED(SYMHSS_K_OTHER, 0.0, launch_copy_blocks(H.D.as<double2>(), H.D.as<double2>(),
                                                    reinterpret_cast<const CopyJob*>(H.cjobs.as<char>() + om),
                                                    (int)mirrors.size(), s));
    // the children's Atilde live in the At buffer one height down
    TIMED(SYMHSS_K_OTHER, 0.0, launch_copy_blocks(h->heights[t - 1].At.as<double2>(), H.D.as<double2>(),
                                                  H.cjobs.as<CopyJob>(), (int)copies.size(), s));
  }
  std::vector<LuJob> lj;
  double lu_work = 0;
  for (size_t b = 0; b < refs.size(); ++b) {
    const HBox& bx = *refs[b].bx;
    LuJob j;
    j.a_off = bx.d_off; j.n = bx.size; j.ld = bx.size; j.piv_off = bx.piv_off;
    j.info_idx = (int)b;
    lj.push_back(j);
    h->st.flops_lu += 8.0 / 3.0 * std::pow((double)bx.size, 3);
    lu_work += 8.0 / 3.0 * std::pow((double)bx.size, 3);
  }
  Packer pk;
  pk.add(lj);
  CK(pk.upload(H.lujobs, s));
  LuLaunch la;
  la.base = H.D.as<double2>();
  la.piv = H.piv.as<int>();
  la.info = H.info.as<int>();
  la.jobs = H.lujobs.as<LuJob>();
  la.njobs = (int)lj.size();
  la.max_n = max_n;
  la.status = h->status.as<int>();
  la.lookahead = h->tune.lu_lookahead;
  la.panel_threads = h->tune.lu_panel_threads;
  la.panel_cluster = h->tune.lu_panel_cluster;
  la.tc = h->tune.lu_tc;
  la.outer = h->tune.lu_outer > 0 ? h->tune.lu_outer : 64;
  la.perm = H.perm.as<int>();
  CK(H.zimg.ensure((size_t)zgemm_lu_img_bytes(la.njobs, max_n)));
  la.zimg = H.zimg.as<unsigned char>();
  la.zimg_bytes = (long long)H.zimg.cap;
  // the assembled blocks are the FP64 operator's (leaf blocks, sibling skeleton blocks)
  CK(H.Dop.ensure(d_total * sizeof(double2)));
  CK(cudaMemcpyAsync(H.Dop.p, H.D.p, d_total * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  if (h->prm.precision == SYMHSS_MIXED) {
    CK(H.D32.ensure(d_total * sizeof(float2)));
    TIMED(SYMHSS_K_OTHER, 0.0, launch_narrow(H.D.as<double2>(), H.D32.as<float2>(), d_total, s));
    la.base32 = H.D32.as<float2>();
    TIMED(SYMHSS_K_GETRF, lu_work, launch_getrf(la, s));
    // LU factors in FP64 for the solve phase
    TIMED(SYMHSS_K_OTHER, 0.0, launch_widen(H.D32.as<float2>(), H.D.as<double2>(), d_total, s));
  } else {
    TIMED(SYMHSS_K_GETRF, lu_work, launch_getrf(la, s));
  }
  return SYMHSS_OK;
}

// lu_done: the height's diagonal blocks were already assembled and factorised (the
// leaf blocks of a pipelined build, which need no compression)
int factor_height(symhss_s* h, int t, cudaStream_t s, long long& pairs, bool lu_done = false) {
  Height& H = h->heights[t];
  int rc = lu_done ? SYMHSS_OK : assemble_and_lu(h, t, s, pairs);
  if (rc) return rc;
  std::vector<BoxRef> refs;
  height_boxes(h, t, false, refs);
  if (refs.empty()) return SYMHSS_OK;
  // bases: L (row ID) for X = D^{-1} L; R (column ID) for R X
  std::vector<int> qhost;
  long long x_total = 0, rx_total = 0, rxpiv_total = 0;
  int max_n = 1, max_k = 1;
  std::vector<int> pos[2], rpos[2];
  for (const BoxRef& rf : refs) {
    HBox& bx = *rf.bx;
    positions(h, t, rf, false, pos);
    positions(h, t, rf, true, rpos);
    for (int p = 0; p < 2; ++p) {
      bx.q_off[p] = (long long)qhost.size();
      for (int c = 0; c < (int)bx.perm[p].size(); ++c) qhost.push_back(pos[p][bx.perm[p][c]]);
      bx.rq_off[p] = (long long)qhost.size();
      for (int c = 0; c < (int)bx.rperm[p].size(); ++c) qhost.push_back(rpos[p][bx.rperm[p][c]]);
    }
    bx.k = bx.rank[0] + bx.rank[1];
    bx.x_off = x_total;
    x_total += (long long)bx.size * bx.k;
    bx.rx_off = rx_total;
    rx_total += (long long)bx.k * bx.k;
    bx.rxpiv_off = rxpiv_total;
    rxpiv_total += bx.k;
    max_n = std::max(max_n, bx.size);
    max_k = std::max(max_k, bx.k);
  }
  // job lists
  std::vector<BasisJob> lbj, rbj;
  std::vector<RsJob> xs, ats;
  std::vector<LuJob> rxl;
  std::vector<CopyJob> eye;
  for (size_t b = 0; b < refs.size(); ++b) {
    HBox& bx = *refs[b].bx;
    BasisJob jl{}, jr{};
    for (int p = 0; p < 2; ++p) {
      jl.part[p].q_off = bx.rq_off[p]; jl.part[p].t_off = bx.rt_off[p];
      jl.part[p].n = (int)bx.rperm[p].size(); jl.part[p].r = bx.rrank[p];
      jl.part[p].col0 = p == 0 ? 0 : bx.rrank[0];
      jr.part[p].q_off = bx.q_off[p]; jr.part[p].t_off = bx.t_off[p];
      jr.part[p].n = (int)bx.perm[p].size(); jr.part[p].r = bx.rank[p];
      jr.part[p].col0 = p == 0 ? 0 : bx.rank[0];
    }
    jl.size = jr.size = bx.size;
    jl.k = jr.k = bx.k;
    jl.out_off = bx.x_off; jl.ld_out = bx.size;
    jr.in_off = bx.x_off; jr.ld_in = bx.size; jr.out_off = bx.rx_off; jr.ld_out = bx.k; jr.ncols = bx.k;
    lbj.push_back(jl);
    rbj.push_back(jr);
    RsJob x;
    x.a_off = bx.d_off; x.n = bx.size; x.lda = bx.size; x.piv_off = bx.piv_off;
    x.b_off = bx.x_off; x.ldb = bx.size; x.nrhs = bx.k;
    xs.push_back(x);
    h->st.flops_lu += 8.0 * (double)bx.size * bx.size * bx.k;
    LuJob lu;
    lu.a_off = bx.rx_off; lu.n = bx.k; lu.ld = bx.k; lu.piv_off = bx.rxpiv_off; lu.info_idx = (int)b;
    rxl.push_back(lu);
    RsJob at;
    at.a_off = bx.rx_off; at.n = bx.k; at.lda = bx.k; at.piv_off = bx.rxpiv_off;
    at.b_off = bx.rx_off; at.ldb = bx.k; at.nrhs = bx.k;
    ats.push_back(at);
    CopyJob cj;
    cj.src_off = -1; cj.dst_off = bx.rx_off; cj.rows = bx.k; cj.cols = bx.k; cj.lds = bx.k; cj.ldd = bx.k;
    eye.push_back(cj);
    h->st.flops_lu += 8.0 / 3.0 * std::pow((double)bx.k, 3) + 8.0 * std::pow((double)bx.k, 3);
  }
  Packer pk;
  const size_t oq = pk.add(qhost), ol = pk.add(lbj), orr = pk.add(rbj), ox = pk.add(xs), orl = pk.add(rxl),
               oa = pk.add(ats), oe = pk.add(eye);
  CK(pk.upload(H.qbuf, s));
  char* qb = H.qbuf.as<char>();
  CK(H.X.ensure(x_total * sizeof(double2)));
  CK(H.RX.ensure(rx_total * sizeof(double2)));
  CK(H.At.ensure(rx_total * sizeof(double2)));
  const bool mixed = h->prm.precision == SYMHSS_MIXED;
  if (mixed) {
    CK(H.X32.ensure(x_total * sizeof(float2)));
    CK(H.RX32.ensure(rx_total * sizeof(float2)));
    CK(H.At32.ensure(rx_total * sizeof(float2)));
  }
  // X = D^{-1} L
  BasisLaunch bl;
  bl.q = reinterpret_cast<const int*>(qb + oq);
  bl.T = H.tbuf.as<double2>();
  bl.in = nullptr;
  bl.out = H.X.as<double2>();
  if (mixed) bl.out32 = H.X32.as<float2>();
  bl.jobs = reinterpret_cast<const BasisJob*>(qb + ol);
  bl.njobs = (int)lbj.size();
  bl.max_cols = max_k;
  TIMED(SYMHSS_K_OTHER, 0.0, launch_basis_dense(bl, s));
  double w_x = 0, w_rx = 0, w_rxlu = 0, w_at = 0;
  for (const BoxRef& rf : refs) {
    const HBox& bx = *rf.bx;
    w_x += 8.0 * (double)bx.size * bx.size * bx.k;
    w_rx += 8.0 * (double)bx.k * bx.k * (double)(bx.perm[0].size() + bx.perm[1].size());
    w_rxlu += 8.0 / 3.0 * std::pow((double)bx.k, 3);
    w_at += 8.0 * std::pow((double)bx.k, 3);
  }
  RsLaunch ra;
  ra.abase = H.D.as<double2>();
  ra.piv = H.piv.as<int>();
  ra.bbase = H.X.as<double2>();
  if (mixed) {
    ra.abase32 = H.D32.as<float2>();
    ra.bbase32 = H.X32.as<float2>();
  }
  ra.jobs = reinterpret_cast<const RsJob*>(qb + ox);
  ra.njobs = (int)xs.size();
  ra.max_rhs = max_k;
  ra.max_n = max_n;
  ra.status = h->status.as<int>();
  ra.tc = h->tune.lu_tc;
  {
    // one scratch for the height's tensor-core products (one stream): the largest of them
    const int nb = (int)refs.size();
    const long long need = std::max({zgemm_lu_img_bytes(nb, max_n), zgemm_rs_img_bytes(nb, max_n, max_k),
                                     zgemm_lu_img_bytes(nb, max_k), zgemm_rs_img_bytes(nb, max_k, max_k)});
    CK(H.zimg.ensure((size_t)need));
  }
  ra.zimg = H.zimg.as<unsigned char>();
  ra.zimg_bytes = (long long)H.zimg.cap;
  {
    // the blocked solves apply their diagonal blocks' inverses on the tensor cores
    CK(H.dinv.ensure((size_t)std::max(getrs_dinv_bytes((int)refs.size(), max_n),
                                       getrs_dinv_bytes((int)refs.size(), max_k))));
    ra.dinv = H.dinv.as<double2>();
    ra.dinv_bytes = (long long)H.dinv.cap;
  }
  ra.perm = H.perm.as<int>();
  TIMED(SYMHSS_K_GETRS, w_x, launch_getrs(ra, s));
  // R X
  BasisLaunch br = bl;
  br.in = H.X.as<double2>();
  br.out = H.RX.as<double2>();
  if (mixed) {
    br.in32 = H.X32.as<float2>();
    br.out32 = H.RX32.as<float2>();
  }
  br.jobs = reinterpret_cast<const BasisJob*>(qb + orr);
  TIMED(SYMHSS_K_OTHER, w_rx, launch_apply_r(br, s));
  // Atilde = (R X)^{-1}
  CK(H.rxpiv.ensure(rxpiv_total * sizeof(int)));
  CK(H.rxperm.ensure(rxpiv_total * sizeof(int)));
  LuLaunch la;
  la.base = H.RX.as<double2>();
  if (mixed) la.base32 = H.RX32.as<float2>();
  la.piv = H.rxpiv.as<int>();
  la.info = H.info.as<int>();
  la.jobs = reinterpret_cast<const LuJob*>(qb + orl);
  la.njobs = (int)rxl.size();
  la.max_n = max_k;
  la.status = h->status.as<int>();
  la.lookahead = h->tune.lu_lookahead;
  la.panel_threads = h->tune.lu_panel_threads;
  la.panel_cluster = h->tune.lu_panel_cluster;
  la.tc = h->tune.lu_tc;
  la.outer = h->tune.lu_outer > 0 ? h->tune.lu_outer : 64;
  la.zimg = H.zimg.as<unsigned char>();
  la.zimg_bytes = (long long)H.zimg.cap;
  la.perm = H.rxperm.as<int>();
  TIMED(SYMHSS_K_GETRF, w_rxlu, launch_getrf(la, s));
  if (mixed)
    TIMED(SYMHSS_K_OTHER, 0.0, launch_copy_blocks32(nullptr, H.At32.as<float2>(),
                                                    reinterpret_cast<const CopyJob*>(qb + oe), (int)eye.size(), s));
  else
    TIMED(SYMHSS_K_OTHER, 0.0, launch_copy_blocks(nullptr, H.At.as<double2>(),
                                                  reinterpret_cast<const CopyJob*>(qb + oe), (int)eye.size(), s));
  RsLaunch rb;
  rb.abase = H.RX.as<double2>();
  rb.piv = H.rxpiv.as<int>();
  rb.bbase = H.At.as<double2>();
  if (mixed) {
    rb.abase32 = H.RX32.as<float2>();
    rb.bbase32 = H.At32.as<float2>();
  }
  rb.jobs = reinterpret_cast<const RsJob*>(qb + oa);
  rb.njobs = (int)ats.size();
  rb.max_rhs = max_k;
  rb.max_n = max_k;
  rb.status = h->status.as<int>();
  rb.tc = h->tune.lu_tc;
  rb.zimg = H.zimg.as<unsigned char>();
  rb.zimg_bytes = (long long)H.zimg.cap;
  rb.dinv = ra.dinv;
  rb.dinv_bytes = ra.dinv_bytes;
  rb.perm = H.rxperm.as<int>();
  TIMED(SYMHSS_K_GETRS, w_at, launch_getrs(rb, s));
  if (mixed) {  // X and Atilde in FP64 for the parents' blocks and the solve phase
    TIMED(SYMHSS_K_OTHER, 0.0, launch_widen(H.X32.as<float2>(), H.X.as<double2>(), x_total, s));
    TIMED(SYMHSS_K_OTHER, 0.0, launch_widen(H.At32.as<float2>(), H.At.as<double2>(), rx_total, s));
  }
  return SYMHSS_OK;
}

// leaf gather / scatter jobs of every leaf of every problem
void leaf_jobs(symhss_s* h, std::vector<LeafJob>& out) {
  out.clear();
  std::vector<BoxRef> refs;
  height_boxes(h, 0, true, refs);
  for (const BoxRef& rf : refs) {
    const Problem& P = h->probs[rf.p];
    const HBox& bx = *rf.bx;
    out.push_back(LeafJob{bx.g_off, P.vec0, bx.begin - P.node0, bx.end - bx.begin, P.n, 0});
  }
}

int validate_params(const symhss_params* p) {
  if (!p) return SYMHSS_ERR_INVALID;
  if (!(p->k0 > 0) || !(p->k1 > 0) || !(p->eps0 > 0) || !(p->eps1 > 0)) return SYMHSS_ERR_INVALID;
  if (!std::isfinite(p->k0) || !std::isfinite(p->k1) || !std::isfinite(p->eps0) || !std::isfinite(p->eps1))
    return SYMHSS_ERR_INVALID;
  if (!(p->tol >= 0) || !std::isfinite(p->tol)) return SYMHSS_ERR_INVALID;
  if (p->leaf < 1 || p->nproxy < 8 || !(p->proxy_factor > 1.0) || !std::isfinite(p->proxy_factor))
    return SYMHSS_ERR_INVALID;
  if (p->mode != SYMHSS_SYM && p->mode != SYMHSS_NONSYM) return SYMHSS_ERR_INVALID;
  if (p->precision != SYMHSS_FP64 && p->precision != SYMHSS_MIXED) return SYMHSS_ERR_INVALID;
  if (p->fixed_rank_kL < 0 || (p->fixed_rank_kL > 0 && !(p->rank_scale_a >= 1.0))) return SYMHSS_ERR_INVALID;
  if (p->oversample < 0) return SYMHSS_ERR_INVALID;
  if (p->formulation != SYMHSS_MULLER && p->formulation != SYMHSS_PMCHWT && p->formulation != SYMHSS_BM)
    return SYMHSS_ERR_INVALID;
  if (p->formulation == SYMHSS_BM && p->mode != SYMHSS_NONSYM) return SYMHSS_ERR_INVALID;
  return SYMHSS_OK;
}

// the fields every problem of a batch must share
bool same_shared(const symhss_params& a, const symhss_params& b) {
  return a.tol == b.tol && a.leaf == b.leaf && a.nproxy == b.nproxy && a.proxy_factor == b.proxy_factor &&
         a.mode == b.mode && a.precision == b.precision && a.fixed_rank_kL == b.fixed_rank_kL &&
         a.rank_scale_a == b.rank_scale_a && a.oversample == b.oversample && a.seed == b.seed &&
         a.formulation == b.formulation;
}

// Copy the curves (host or device arrays) into the concatenated host node arrays.
int load_curves(symhss_s* h, const symhss_curve* cs, int count, cudaStream_t s) {
  long long total = 0;
  for (int c = 0; c < count; ++c) {
    const symhss_curve* cv = &cs[c];
    if (cv->n < 2) return SYMHSS_ERR_INVALID;
    if (!cv->x || !cv->y || !cv->nx || !cv->ny || !cv->w || !cv->kappa) return SYMHSS_ERR_INVALID;
    if (cv->location != SYMHSS_HOST && cv->location != SYMHSS_DEVICE) return SYMHSS_ERR_INVALID;
    total += cv->n;
  }
  if (total > (1LL << 30)) return SYMHSS_ERR_INVALID;
  std::vector<double>* dst[6] = {&h->hx, &h->hy, &h->hnx, &h->hny, &h->hw, &h->hk};
  for (int i = 0; i < 6; ++i) dst[i]->resize((size_t)total);
  bool any_device = false;
  long long off = 0;
  for (int c = 0; c < count; ++c) {
    const symhss_curve* cv = &cs[c];
    const double* src[6] = {cv->x, cv->y, cv->nx, cv->ny, cv->w, cv->kappa};
    for (int i = 0; i < 6; ++i) {
      double* d = dst[i]->data() + off;
      if (cv->location == SYMHSS_HOST) {
        std::memcpy(d, src[i], cv->n * sizeof(double));
      } else {
        any_device = true;
        cudaError_t e = cudaMemcpyAsync(d, src[i], cv->n * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(h, e);
      }
    }
    off += cv->n;
  }
  if (any_device) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e);
  }
  for (int i = 0; i < 6; ++i)
    if (!finite_all(*dst[i])) return SYMHSS_ERR_INVALID;
  for (long long i = 0; i < total; ++i)
    if (!(h->hw[i] > 0)) return SYMHSS_ERR_INVALID;
  for (int c = 0; c < count; ++c) h->probs[c].n = cs[c].n;
  return SYMHSS_OK;
}

void geometry_stats(symhss_s* h) {
  h->st.n = h->ntot;
  h->st.depth = h->maxdepth;
  int leaves = 0;
  for (const Problem& P : h->probs) leaves += (int)P.levels[P.depth].size();
  h->st.nboxes_leaf = leaves;
}

}  // namespace
}  // namespace symhss

using namespace symhss;

// =============================================================================== C ABI

extern "C" {

const char* symhss_strerror(int status) {
  switch (status) {
    case SYMHSS_OK: return "ok";
    case SYMHSS_ERR_INVALID: return "invalid argument";
    case SYMHSS_ERR_NOMEM: return "out of memory";
    case SYMHSS_ERR_CUDA: return "CUDA error";
    case SYMHSS_ERR_RANK_OVERFLOW: return "ID rank exceeded capacity";
    case SYMHSS_ERR_SINGULAR: return "singular diagonal block";
    case SYMHSS_ERR_TIMEOUT: return "device wait timed out";
    case SYMHSS_ERR_STATE: return "calls out of order";
    case SYMHSS_ERR_DEVICE: return "device-side index check failed";
    default: return "unknown status";
  }
}

int symhss_params_default(symhss_params* p) {
  if (!p) return SYMHSS_ERR_INVALID;
  std::memset(p, 0, sizeof(*p));
  p->k0 = 1.0; p->k1 = 1.0; p->eps0 = 1.0; p->eps1 = 1.0;
  p->tol = 1e-10; p->leaf = 128; p->nproxy = 64; p->proxy_factor = 1.5;
  p->mode = SYMHSS_SYM; p->precision = SYMHSS_FP64;
  p->fixed_rank_kL = 0; p->rank_scale_a = 1.15; p->oversample = 16; p->seed = 0x5eed;
  return SYMHSS_OK;
}

int symhss_create_batch(const symhss_curve* curves, const symhss_params* prms, int count, void* stream,
                        symhss_t* out) {
  if (!out) return SYMHSS_ERR_INVALID;
  *out = nullptr;
  if (!curves || !prms || count < 1) return SYMHSS_ERR_INVALID;
  for (int c = 0; c < count; ++c) {
    int rc = validate_params(&prms[c]);
    if (rc) return rc;
    if (!same_shared(prms[0], prms[c])) return SYMHSS_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  symhss_s* h = new (std::nothrow) symhss_s();
  if (!h) return SYMHSS_ERR_NOMEM;
  int rc = SYMHSS_OK;
  try {
    h->prm = prms[0];
    h->probs.resize(count);
    for (int c = 0; c < count; ++c) h->probs[c].prm = prms[c];
    rc = load_curves(h, curves, count, s);
    if (!rc) rc = build_geometry(h, s);
    if (!rc) {
      cudaError_t e = h->status.ensure(sizeof(int));
      if (e == cudaSuccess) e = cudaMemsetAsync(h->status.p, 0, sizeof(int), s);
      for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreate(&h->ev[i]);
      if (e != cudaSuccess) rc = cuda_fail(h, e);
    }
  } catch (const std::bad_alloc&) {
    rc = SYMHSS_ERR_NOMEM;
  }
  if (rc) {
    symhss_destroy(h);
    return rc;
  }
  geometry_stats(h);
  *out = h;
  return SYMHSS_OK;
}

int symhss_create(const symhss_curve* curve, const symhss_params* prm, void* stream, symhss_t* out) {
  if (!curve || !prm) {
    if (out) *out = nullptr;
    return SYMHSS_ERR_INVALID;
  }
  return symhss_create_batch(curve, prm, 1, stream, out);
}

int symhss_set_curves(symhss_t h, const symhss_curve* curves, int count, void* stream) {
  BudgetScope budget_scope(h ? &h->budget : nullptr);
  if (!h || !curves || count != (int)h->probs.size()) return SYMHSS_ERR_INVALID;
  for (int c = 0; c < count; ++c)
    if (curves[c].n != h->probs[c].n) return SYMHSS_ERR_INVALID;
  try {
    h->compressed = h->factored = false;
    int rc = load_curves(h, curves, count, (cudaStream_t)stream);
    if (rc) return rc;
    rc = build_geometry(h, (cudaStream_t)stream);
    if (!rc) geometry_stats(h);
    return rc;
  } catch (const std::bad_alloc&) {
    return SYMHSS_ERR_NOMEM;
  }
}

int symhss_set_curve(symhss_t h, const symhss_curve* curve, void* stream) {
  if (!h || (int)h->probs.size() != 1) return SYMHSS_ERR_INVALID;
  return symhss_set_curves(h, curve, 1, stream);
}

int symhss_batch_info(symhss_t h, int* count, int* n, int* depth, long long* row0) {
  if (!h) return SYMHSS_ERR_INVALID;
  if (count) *count = (int)h->probs.size();
  for (size_t c = 0; c < h->probs.size(); ++c) {
    if (n) n[c] = h->probs[c].n;
    if (depth) depth[c] = h->probs[c].depth;
    if (row0) row0[c] = h->probs[c].vec0;
  }
  return SYMHSS_OK;
}

static void reset_compress_stats(symhss_s* h) {
  h->compressed = h->factored = false;
  h->st.ms_tiles = h->st.ms_id = 0;
  h->st.pairs_evaluated = 0;
  h->st.id_count = 0;
  h->st.flops_id = 0;
  h->st.sketch_redo = 0;
  h->st.check_failed = 0;
  h->st.check_max_ratio = 0;
  h->st.proposals = 0;
  h->st.proposal_rank_err = 0;
  h->st.proposal_under = 0;
  for (int c = 0; c < SYMHSS_K_COUNT; ++c) {
    h->st.kernel_ms[c] = 0;
    h->st.kernel_launches[c] = 0;
    h->st.kernel_work[c] = 0;
  }
  h->marks.clear();
  h->evnext = 0;
}

static void rank_stats(symhss_s* h) {
  // rank statistics by level, over every problem that has the level
  h->st.max_rank[0] = h->st.max_rank[1] = 0;
  for (int l = 0; l < SYMHSS_MAX_LEVELS; ++l) {
    h->st.level_nproxy[l] = 0;
    for (int p = 0; p < 2; ++p) {
      h->st.level_max_rank[l][p] = 0;
      h->st.level_mean_rank[l][p] = 0.0;
    }
  }
  for (int l = 1; l <= h->maxdepth; ++l) {
    for (int p = 0; p < 2; ++p) {
      int mx = 0;
      double sum = 0;
      long long cnt = 0;
      for (const Problem& P : h->probs) {
        if (P.depth < l) continue;
        for (const HBox& b : P.levels[l]) { mx = std::max(mx, b.rank[p]); sum += b.rank[p]; ++cnt; }
      }
      h->st.level_max_rank[l][p] = mx;
      h->st.level_mean_rank[l][p] = cnt ? sum / (double)cnt : 0.0;
      h->st.max_rank[p] = std::max(h->st.max_rank[p], mx);
    }
    int mp = 0;
    for (const Problem& P : h->probs)
      if (P.depth >= l)
        for (const HBox& b : P.levels[l]) mp = std::max(mp, b.P);
    h->st.level_nproxy[l] = mp;
  }
}

int symhss_compress(symhss_t h, void* stream) {
  BudgetScope budget_scope(h ? &h->budget : nullptr);
  if (!h) return SYMHSS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  reset_compress_stats(h);
  try {
    CK(cudaMemsetAsync(h->status.p, 0, sizeof(int), s));
    CK(cudaEventRecord(h->ev[0], s));
    for (int t = 0; t < h->maxdepth; ++t) {
      int rc = compress_height(h, t, s);
      if (rc) return rc;
      rc = read_status(h, s);
      if (rc) return rc;
    }
    CK(cudaEventRecord(h->ev[1], s));
    CK(cudaEventSynchronize(h->ev[1]));
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
    h->st.ms_compress = ms;
    if (h->st.proposals > 0) h->st.proposal_rank_err /= (double)h->st.proposals;
  } catch (const std::bad_alloc&) {
    return SYMHSS_ERR_NOMEM;
  }
  rank_stats(h);
  h->compressed = true;
  return SYMHSS_OK;
}

int symhss_factor(symhss_t h, void* stream) {
  BudgetScope budget_scope(h ? &h->budget : nullptr);
  if (!h) return SYMHSS_ERR_INVALID;
  if (!h->compressed && h->maxdepth > 0) return SYMHSS_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  h->factored = false;
  h->st.flops_lu = 0;
  long long pairs = 0;
  try {
    CK(cudaMemsetAsync(h->status.p, 0, sizeof(int), s));
    CK(cudaEventRecord(h->ev[0], s));
    for (int t = 0; t <= h->maxdepth; ++t) {
      int rc = factor_height(h, t, s, pairs);
      if (rc) return rc;
    }
    CK(cudaEventRecord(h->ev[1], s));
    int rc = read_status(h, s);
    if (rc) return rc;
    prof_collect(h);
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
    h->st.ms_factor = ms;
    int rs = 0;
    for (const Problem& P : h->probs) rs = std::max(rs, P.levels[0][0].size);
    h->st.root_size = rs;
  } catch (const std::bad_alloc&) {
    return SYMHSS_ERR_NOMEM;
  }
  h->st.pairs_evaluated += pairs;
  h->factored = true;
  return SYMHSS_OK;
}

int symhss_build(symhss_t h, void* stream) {
  BudgetScope budget_scope(h ? &h->budget : nullptr);
  if (!h) return SYMHSS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (!h->cstream) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&h->cstream, cudaStreamNonBlocking, hi) != cudaSuccess) {
      cudaGetLastError();
      h->cstream = nullptr;
    }
  }
  if (!h->cstream) {  // no second stream: the two phases one after the other
    int rc = symhss_compress(h, stream);
    return rc ? rc : symhss_factor(h, stream);
  }
  cudaStream_t cs = h->cstream;
  reset_compress_stats(h);
  h->st.flops_lu = 0;
  h->st.ms_compress = h->st.ms_factor = 0;
  long long pairs = 0;
  try {
    CK(cudaMemsetAsync(h->status.p, 0, sizeof(int), s));
    CK(cudaEventRecord(h->ev[0], s));
    CK(cudaStreamWaitEvent(cs, h->ev[0], 0));  // the compression follows earlier work on s
    // the leaf blocks' assembly and LU need no compression: queued first on s, they run
    // while height 0 is compressed on cs
    int rc = assemble_and_lu(h, 0, s, pairs);
    if (rc) return rc;
    if (h->maxdepth > 0) {
      rc = compress_height(h, 0, cs);
      if (!rc) rc = read_status(h, cs);
      if (rc) return rc;
    }
    for (int t = 0; t <= h->maxdepth; ++t) {
      // height t is compressed (its stream was synchronised): factor it on s while the
      // next height is compressed on cs
      rc = factor_height(h, t, s, pairs, t == 0);
      if (rc) return rc;
      if (t + 1 < h->maxdepth) {
        rc = compress_height(h, t + 1, cs);
        if (!rc) rc = read_status(h, cs);
        if (rc) return rc;
      }
    }
    CK(cudaEventRecord(h->ev[1], s));
    rc = read_status(h, s);
    if (rc) return rc;
    CK(cudaStreamSynchronize(cs));
    prof_collect(h);
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
    h->st.ms_build = ms;
    if (h->st.proposals > 0) h->st.proposal_rank_err /= (double)h->st.proposals;
    int rs = 0;
    for (const Problem& P : h->probs) rs = std::max(rs, P.levels[0][0].size);
    h->st.root_size = rs;
  } catch (const std::bad_alloc&) {
    return SYMHSS_ERR_NOMEM;
  }
  rank_stats(h);
  h->st.pairs_evaluated += pairs;
  h->compressed = h->factored = true;
  return SYMHSS_OK;
}

int symhss_rhs_plane_wave(symhss_t h, double angle, void* rhs, void* stream) {
  BudgetScope budget_scope(h ? &h->budget : nullptr);
  if (!h || !rhs || !std::isfinite(angle)) return SYMHSS_ERR_INVALID;
  CK(launch_plane_wave(table_of(h), h->waves.as<WaveJob>(), (int)h->probs.size(), h->max_n, angle,
                       h->prm.mode == SYMHSS_SYM ? 1 : 0, reinterpret_cast<double2*>(rhs), (cudaStream_t)stream));
  return SYMHSS_OK;
}

}  // extern "C"

namespace symhss {
namespace {

// One application of the factorisation's inverse: x = B^{-1} f (Sec. 4.2 up / down pass).
int gemm_max_m(const std::vector<GemmJob>& jobs) {
  int m = 0;
  for (const GemmJob& j : jobs) m = std::max(m, j.m);
  return m;
}

int solve_core(symhss_s* h, const double2* f, double2* xo, int nrhs, cudaStream_t s) {
  const long long ldv = 2LL * h->ntot;
  (void)ldv;
    std::vector<BoxRef> refs;
  // up pass: g = D^{-1} f, f~ = Atilde R g, from the leaves to every root
  for (int t = 0; t <= h->maxdepth; ++t) {
    Height& H = h->heights[t];
    height_boxes(h, t, true, refs);
    if (refs.empty()) continue;
    long long g_total = 0, ft_total = 0;
    for (const BoxRef& rf : refs) {
      HBox& bx = *rf.bx;
      const bool root = rf.l == 0;
      bx.g_off = g_total;
      g_total += (long long)bx.size * nrhs;
      bx.ft_off = ft_total;
      ft_total += (long long)(root ? 0 : bx.k) * nrhs;
    }
    CK(H.G.ensure(g_total * sizeof(double2)));
    CK(H.FT.ensure(ft_total * sizeof(double2)));
    CK(H.TMP.ensure(ft_total * sizeof(double2)));
    Packer pk;
    std::vector<LeafJob> lj;
    std::vector<CopyJob> cj;
    std::vector<RsJob> rs;
    std::vector<BasisJob> bj;
    std::vector<GemmJob> gj;
    int max_n = 1;
    if (t == 0) leaf_jobs(h, lj);
    for (const BoxRef& rf : refs) {
      const HBox& bx = *rf.bx;
      if (t > 0) {
        const auto& kids = h->probs[rf.p].levels[rf.l + 1];
        const HBox& c1 = kids[bx.child[0]];
        const HBox& c2 = kids[bx.child[1]];
        CopyJob c;
        c.src_off = c1.ft_off; c.dst_off = bx.g_off; c.rows = c1.k; c.cols = nrhs; c.lds = c1.k; c.ldd = bx.size;
        cj.push_back(c);
        c.src_off = c2.ft_off; c.dst_off = bx.g_off + c1.k; c.rows = c2.k; c.lds = c2.k;
        cj.push_back(c);
      }
      RsJob r;
      r.a_off = bx.d_off; r.n = bx.size; r.lda = bx.size; r.piv_off = bx.piv_off;
      r.b_off = bx.g_off; r.ldb = bx.size; r.nrhs = nrhs;
      rs.push_back(r);
      max_n = std::max(max_n, bx.size);
      if (rf.l > 0) {
        BasisJob b{};
        for (int p = 0; p < 2; ++p) {
          b.part[p].q_off = bx.q_off[p]; b.part[p].t_off = bx.t_off[p];
          b.part[p].n = (int)bx.perm[p].size(); b.part[p].r = bx.rank[p];
          b.part[p].col0 = p == 0 ? 0 : bx.rank[0];
        }
        b.size = bx.size; b.k = bx.k;
        b.in_off = bx.g_off; b.ld_in = bx.size; b.out_off = bx.ft_off; b.ld_out = bx.k; b.ncols = nrhs;
        bj.push_back(b);
        GemmJob gmm;
        gmm.a_off = bx.rx_off; gmm.lda = bx.k;
        gmm.b_off = bx.ft_off; gmm.ldb = bx.k;
        gmm.c_off = bx.ft_off; gmm.ldc = bx.k;
        gmm.m = bx.k; gmm.n = nrhs; gmm.k = bx.k; gmm.alpha = 1.0; gmm.beta = 0.0;
        gj.push_back(gmm);
      }
    }
    const size_t olj = pk.add(lj), ocj = pk.add(cj), ors = pk.add(rs), obj = pk.add(bj), ogj = pk.add(gj);
    CK(pk.upload(H.slists, s));
    char* sb = H.slists.as<char>();
    if (t == 0)
      TIMED(SYMHSS_K_OTHER, 0.0, launch_leaf_gather(f, ldv, H.G.as<double2>(),
                                                    reinterpret_cast<const LeafJob*>(sb + olj), (int)lj.size(),
                                                    nrhs, s));
    else
      TIMED(SYMHSS_K_OTHER, 0.0, launch_copy_blocks(h->heights[t - 1].FT.as<double2>(), H.G.as<double2>(),
                                                    reinterpret_cast<const CopyJob*>(sb + ocj), (int)cj.size(),
                                                    s));
    double w_g = 0, w_up = 0;
    for (const BoxRef& rf : refs) {
      const HBox& bx = *rf.bx;
      w_g += 8.0 * (double)bx.size * bx.size * nrhs;
      if (rf.l > 0) w_up += 8.0 * (double)bx.k * (double)(bx.perm[0].size() + bx.perm[1].size() + bx.k) * nrhs;
    }
    RsLaunch ra;
    ra.abase = H.D.as<double2>(); ra.piv = H.piv.as<int>(); ra.bbase = H.G.as<double2>();
    ra.jobs = reinterpret_cast<const RsJob*>(sb + ors); ra.njobs = (int)rs.size();
    ra.max_rhs = nrhs; ra.max_n = max_n;
    ra.perm = H.perm.as<int>();
    TIMED(SYMHSS_K_GETRS, w_g, launch_getrs(ra, s));
    if (!bj.empty()) {
      // tmp = R g ; f~ = Atilde tmp
      BasisLaunch ba;
      ba.q = reinterpret_cast<const int*>(H.qbuf.p);
      ba.T = H.tbuf.as<double2>();
      ba.in = H.G.as<double2>();
      ba.out = H.TMP.as<double2>();
      ba.jobs = reinterpret_cast<const BasisJob*>(sb + obj);
      ba.njobs = (int)bj.size();
      ba.max_cols = nrhs;
      TIMED(SYMHSS_K_OTHER, w_up, launch_apply_r(ba, s));
      GemmLaunch ga;
      ga.A = H.At.as<double2>(); ga.B = H.TMP.as<double2>(); ga.C = H.FT.as<double2>();
      ga.jobs = reinterpret_cast<const GemmJob*>(sb + ogj); ga.njobs = (int)gj.size();
      ga.max_m = gemm_max_m(gj); ga.max_n = nrhs;
      TIMED(SYMHSS_K_OTHER, 0.0, launch_gemm(ga, s));
    }
  }
  // down pass: x_c = g_c - X_c (f~_c - Atilde_c y_c), parents at height t + 1
  for (int t = h->maxdepth - 1; t >= 0; --t) {
    Height& H = h->heights[t];
    Height& HP = h->heights[t + 1];
    std::vector<GemmJob> g1, g2;
    for (Problem& P : h->probs) {
      if (P.depth <= t) continue;
      const int l = P.depth - t;
      for (const HBox& par : P.levels[l - 1]) {
        int row0 = 0;
        for (int c = 0; c < 2; ++c) {
          const HBox& bx = P.levels[l][par.child[c]];
          GemmJob a;
          a.a_off = bx.rx_off; a.lda = bx.k;
          a.b_off = par.g_off + row0; a.ldb = par.size;
          a.c_off = bx.ft_off; a.ldc = bx.k;
          a.m = bx.k; a.n = nrhs; a.k = bx.k; a.alpha = -1.0; a.beta = 1.0;
          g1.push_back(a);
          GemmJob b;
          b.a_off = bx.x_off; b.lda = bx.size;
          b.b_off = bx.ft_off; b.ldb = bx.k;
          b.c_off = bx.g_off; b.ldc = bx.size;
          b.m = bx.size; b.n = nrhs; b.k = bx.k; b.alpha = -1.0; b.beta = 1.0;
          g2.push_back(b);
          row0 += bx.k;
        }
      }
    }
    if (g1.empty()) continue;
    Packer pk;
    const size_t o1 = pk.add(g1), o2 = pk.add(g2);
    CK(pk.upload(H.slists, s));
    char* sb = H.slists.as<char>();
    GemmLaunch ga;
    ga.A = H.At.as<double2>(); ga.B = HP.G.as<double2>(); ga.C = H.FT.as<double2>();
    ga.jobs = reinterpret_cast<const GemmJob*>(sb + o1); ga.njobs = (int)g1.size();
    ga.max_m = gemm_max_m(g1); ga.max_n = nrhs;
    double w_dn = 0;
    for (const auto& j : g1) w_dn += 8.0 * (double)j.m * j.n * j.k;
    for (const auto& j : g2) w_dn += 8.0 * (double)j.m * j.n * j.k;
    TIMED(SYMHSS_K_OTHER, w_dn, launch_gemm(ga, s));
    GemmLaunch gb;
    gb.A = H.X.as<double2>(); gb.B = H.FT.as<double2>(); gb.C = H.G.as<double2>();
    gb.jobs = reinterpret_cast<const GemmJob*>(sb + o2); gb.njobs = (int)g2.size();
    gb.max_m = gemm_max_m(g2); gb.max_n = nrhs;
    TIMED(SYMHSS_K_OTHER, 0.0, launch_gemm(gb, s));
  }
  {
    // the leaf lists of height 0 were overwritten by the down pass: upload them again
    std::vector<LeafJob> lj;
    leaf_jobs(h, lj);
    Packer pk;
    const size_t o = pk.add(lj);
    Height& H0 = h->heights[0];
    DevBuf& lb = h->maxdepth > 0 ? h->heights[h->maxdepth].slists : H0.slists;
    CK(pk.upload(lb, s));
    TIMED(SYMHSS_K_OTHER, 0.0, launch_leaf_scatter(H0.G.as<double2>(), xo, ldv,
                           reinterpret_cast<const LeafJob*>(lb.as<char>() + o), (int)lj.size(), nrhs, s));
  }
  return SYMHSS_OK;
}

// y = A_hss x with the kept FP64 blocks and the ID interpolation operators: an up pass of
// skeleton values (xs = R xv), the sibling skeleton blocks at every parent (zv = D_off xv),
// a down pass (yv = zv + L ys_parent; ys_child = rows of yv) and the leaf blocks.
int matvec_core(symhss_s* h, const double2* xin, double2* yout, int nrhs, cudaStream_t s) {
  const long long ldv = 2LL * h->ntot;
  std::vector<BoxRef> refs;
  // offsets: size-sized and k-sized vectors per box and height
  for (int t = 0; t <= h->maxdepth; ++t) {
    Height& H = h->heights[t];
    height_boxes(h, t, true, refs);
    long long v_total = 0, k_total = 0;
    for (const BoxRef& rf : refs) {
      HBox& bx = *rf.bx;
      bx.g_off = v_total;
      v_total += (long long)bx.size * nrhs;
      bx.ft_off = k_total;
      k_total += (long long)(rf.l == 0 ? 0 : bx.k) * nrhs;
    }
    for (DevBuf* b : {&H.XV, &H.ZV, &H.YV}) CK(b->ensure(v_total * sizeof(double2)));
    for (DevBuf* b : {&H.XS, &H.YS}) CK(b->ensure(k_total * sizeof(double2)));
  }
  // up pass
  for (int t = 0; t <= h->maxdepth; ++t) {
    Height& H = h->heights[t];
    height_boxes(h, t, true, refs);
    if (refs.empty()) continue;
    std::vector<LeafJob> lj;
    std::vector<CopyJob> cj;
    std::vector<BasisJob> bj;
    std::vector<GemmJob> gj;
    if (t == 0) leaf_jobs(h, lj);
    for (const BoxRef& rf : refs) {
      const HBox& bx = *rf.bx;
      if (t > 0) {
        const auto& kids = h->probs[rf.p].levels[rf.l + 1];
        const HBox& c1 = kids[bx.child[0]];
        const HBox& c2 = kids[bx.child[1]];
        CopyJob c;
        c.src_off = c1.ft_off; c.dst_off = bx.g_off; c.rows = c1.k; c.cols = nrhs; c.lds = c1.k; c.ldd = bx.size;
        cj.push_back(c);
        c.src_off = c2.ft_off; c.dst_off = bx.g_off + c1.k; c.rows = c2.k; c.lds = c2.k;
        cj.push_back(c);
        // sibling skeleton blocks of the parent: zv = [0 D12; D21 0] xv
        GemmJob g;
        g.a_off = bx.d_off + (long long)c1.k * bx.size; g.lda = bx.size;
        g.b_off = bx.g_off + c1.k; g.ldb = bx.size;
        g.c_off = bx.g_off; g.ldc = bx.size;
        g.m = c1.k; g.n = nrhs; g.k = c2.k; g.alpha = 1.0; g.beta = 0.0;
        gj.push_back(g);
        g.a_off = bx.d_off + c1.k; g.b_off = bx.g_off; g.c_off = bx.g_off + c1.k;
        g.m = c2.k; g.k = c1.k;
        gj.push_back(g);
      } else {
        // leaf block: zv = D xv (the down pass adds L ys)
        GemmJob g;
        g.a_off = bx.d_off; g.lda = bx.size; g.b_off = bx.g_off; g.ldb = bx.size;
        g.c_off = bx.g_off; g.ldc = bx.size; g.m = bx.size; g.n = nrhs; g.k = bx.size;
        g.alpha = 1.0; g.beta = 0.0;
        gj.push_back(g);
      }
      if (rf.l > 0) {
        BasisJob b{};
        for (int p = 0; p < 2; ++p) {
          b.part[p].q_off = bx.q_off[p]; b.part[p].t_off = bx.t_off[p];
          b.part[p].n = (int)bx.perm[p].size(); b.part[p].r = bx.rank[p];
          b.part[p].col0 = p == 0 ? 0 : bx.rank[0];
        }
        b.size = bx.size; b.k = bx.k;
        b.in_off = bx.g_off; b.ld_in = bx.size; b.out_off = bx.ft_off; b.ld_out = bx.k; b.ncols = nrhs;
        bj.push_back(b);
      }
    }
    Packer pk;
    const size_t olj = pk.add(lj), ocj = pk.add(cj), obj = pk.add(bj), ogj = pk.add(gj);
    CK(pk.upload(H.mlists, s));
    char* sb = H.mlists.as<char>();
    if (t == 0)
      CK(launch_leaf_gather(xin, ldv, H.XV.as<double2>(), reinterpret_cast<const LeafJob*>(sb + olj), (int)lj.size(),
                            nrhs, s));
    else
      CK(launch_copy_blocks(h->heights[t - 1].XS.as<double2>(), H.XV.as<double2>(),
                            reinterpret_cast<const CopyJob*>(sb + ocj), (int)cj.size(), s));
    GemmLaunch ga;
    ga.A = H.Dop.as<double2>(); ga.B = H.XV.as<double2>(); ga.C = H.ZV.as<double2>();
    ga.jobs = reinterpret_cast<const GemmJob*>(sb + ogj); ga.njobs = (int)gj.size();
    ga.max_m = gemm_max_m(gj); ga.max_n = nrhs;
    CK(launch_gemm(ga, s));
    if (!bj.empty()) {
      BasisLaunch ba;
      ba.q = reinterpret_cast<const int*>(H.qbuf.p);
      ba.T = H.tbuf.as<double2>();
      ba.in = H.XV.as<double2>();
      ba.out = H.XS.as<double2>();
      ba.jobs = reinterpret_cast<const BasisJob*>(sb + obj);
      ba.njobs = (int)bj.size();
      ba.max_cols = nrhs;
      CK(launch_apply_r(ba, s));
    }
  }
  // down pass: yv = zv + L ys (non-root), children's ys = their rows of yv
  for (int t = h->maxdepth; t >= 0; --t) {
    Height& H = h->heights[t];
    height_boxes(h, t, true, refs);
    if (refs.empty()) continue;
    std::vector<BasisJob> lbj;
    std::vector<CopyJob> cz, cd;
    for (const BoxRef& rf : refs) {
      const HBox& bx = *rf.bx;
      CopyJob c;
      c.src_off = bx.g_off; c.dst_off = bx.g_off; c.rows = bx.size; c.cols = nrhs; c.lds = bx.size; c.ldd = bx.size;
      cz.push_back(c);
      if (rf.l > 0) {
        BasisJob b{};
        for (int p = 0; p < 2; ++p) {
          b.part[p].q_off = bx.rq_off[p]; b.part[p].t_off = bx.rt_off[p];
          b.part[p].n = (int)bx.rperm[p].size(); b.part[p].r = bx.rrank[p];
          b.part[p].col0 = p == 0 ? 0 : bx.rrank[0];
        }
        b.size = bx.size; b.k = bx.k;
        b.in_off = bx.ft_off; b.ld_in = bx.k; b.out_off = bx.g_off; b.ld_out = bx.size; b.ncols = nrhs;
        lbj.push_back(b);
      }
      if (t > 0) {
        const auto& kids = h->probs[rf.p].levels[rf.l + 1];
        const HBox& c1 = kids[bx.child[0]];
        const HBox& c2 = kids[bx.child[1]];
        c.src_off = bx.g_off; c.dst_off = c1.ft_off; c.rows = c1.k; c.cols = nrhs; c.lds = bx.size; c.ldd = c1.k;
        cd.push_back(c);
        c.src_off = bx.g_off + c1.k; c.dst_off = c2.ft_off; c.rows = c2.k; c.lds = bx.size; c.ldd = c2.k;
        cd.push_back(c);
      }
    }
    Packer pk;
    const size_t ol = pk.add(lbj), oz = pk.add(cz), od = pk.add(cd);
    CK(pk.upload(H.mlists, s));
    char* sb = H.mlists.as<char>();
    // yv = zv (+ L ys)
    CK(launch_copy_blocks(H.ZV.as<double2>(), H.YV.as<double2>(), reinterpret_cast<const CopyJob*>(sb + oz),
                          (int)cz.size(), s));
    if (!lbj.empty()) {
      BasisLaunch bl;
      bl.q = reinterpret_cast<const int*>(H.qbuf.p);
      bl.T = H.tbuf.as<double2>();
      bl.in = H.YS.as<double2>();
      bl.out = H.YV.as<double2>();
      bl.jobs = reinterpret_cast<const BasisJob*>(sb + ol);
      bl.njobs = (int)lbj.size();
      bl.max_cols = nrhs;
      CK(launch_apply_l(bl, s));  // yv += L ys
    }
    if (t > 0)
      CK(launch_copy_blocks(H.YV.as<double2>(), h->heights[t - 1].YS.as<double2>(),
                            reinterpret_cast<const CopyJob*>(sb + od), (int)cd.size(), s));
  }
  {
    std::vector<LeafJob> lj;
    leaf_jobs(h, lj);
    Packer pk;
    const size_t o = pk.add(lj);
    DevBuf& lb = h->maxdepth > 0 ? h->heights[h->maxdepth].mlists : h->heights[0].mlists;
    CK(pk.upload(lb, s));
    CK(launch_leaf_scatter(h->heights[0].YV.as<double2>(), yout, ldv,
                           reinterpret_cast<const LeafJob*>(lb.as<char>() + o), (int)lj.size(), nrhs, s));
  }
  return SYMHSS_OK;
}

}  // namespace
}  // namespace symhss

extern "C" {

int symhss_solve(symhss_t h, const void* rhs, void* x, int nrhs, void* stream) {
  BudgetScope budget_scope(h ? &h->budget : nullptr);
  if (!h || !rhs || !x || nrhs < 1) return SYMHSS_ERR_INVALID;
  if (!h->factored) return SYMHSS_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  const double2* f = reinterpret_cast<const double2*>(rhs);
  double2* xo = reinterpret_cast<double2*>(x);
  try {
    CK(cudaEventRecord(h->ev[0], s));
    int rc = solve_core(h, f, xo, nrhs, s);
    if (rc) return rc;
    if (h->prm.precision == SYMHSS_MIXED && h->refine_steps > 0) {
      // x <- x + B^{-1} (f - A_hss x), A_hss the FP64 compressed operator
      const long long len = 2LL * h->ntot * nrhs;
      CK(h->rres.ensure(len * sizeof(double2)));
      CK(h->rcor.ensure(len * sizeof(double2)));
      for (int it = 0; it < h->refine_steps; ++it) {
        rc = matvec_core(h, xo, h->rres.as<double2>(), nrhs, s);
        if (rc) return rc;
        TIMED(SYMHSS_K_OTHER, 0.0, launch_axpby(f, h->rres.as<double2>(), len, 1.0, -1.0, s));
        rc = solve_core(h, h->rres.as<double2>(), h->rcor.as<double2>(), nrhs, s);
        if (rc) return rc;
        TIMED(SYMHSS_K_OTHER, 0.0, launch_axpby(h->rcor.as<double2>(), xo, len, 1.0, 1.0, s));
      }
    }
    CK(cudaEventRecord(h->ev[1], s));
    rc = read_status(h, s);
    if (rc) return rc;
    prof_collect(h);
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
    h->st.ms_solve = ms;
  } catch (const std::bad_alloc&) {
    return SYMHSS_ERR_NOMEM;
  }
  return SYMHSS_OK;
}

int symhss_matvec(symhss_t h, const void* x, void* y, int nrhs, void* stream) {
  BudgetScope budget_scope(h ? &h->budget : nullptr);
  if (!h || !x || !y || nrhs < 1) return SYMHSS_ERR_INVALID;
  if (!h->factored) return SYMHSS_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    int rc = matvec_core(h, reinterpret_cast<const double2*>(x), reinterpret_cast<double2*>(y), nrhs, s);
    if (rc) return rc;
    CK(cudaStreamSynchronize(s));
  } catch (const std::bad_alloc&) {
    return SYMHSS_ERR_NOMEM;
  }
  return SYMHSS_OK;
}

int symhss_set_refinement(symhss_t h, int steps) {
  if (!h || steps < 0 || steps > 4) return SYMHSS_ERR_INVALID;
  h->refine_steps = steps;
  return SYMHSS_OK;
}

int symhss_solve_host(symhss_t h, const void* rhs_host, void* x_host, int nrhs, void* stream) {
  BudgetScope budget_scope(h ? &h->budget : nullptr);
  if (!h || !rhs_host || !x_host || nrhs < 1) return SYMHSS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)2 * h->ntot * nrhs * sizeof(double2);
  CK(h->xin.ensure(bytes));
  CK(h->xout.ensure(bytes));
  CK(cudaMemcpyAsync(h->xin.p, rhs_host, bytes, cudaMemcpyHostToDevice, s));
  int rc = symhss_solve(h, h->xin.p, h->xout.p, nrhs, stream);
  if (rc) return rc;
  CK(cudaMemcpyAsync(x_host, h->xout.p, bytes, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return SYMHSS_OK;
}

int symhss_stats(symhss_t h, symhss_stats_t* out) {
  if (!h || !out) return SYMHSS_ERR_INVALID;
  long long bytes = (long long)h->pts.cap + (long long)h->status.cap + h->xin.cap + h->xout.cap + h->kps.cap +
                    h->waves.cap + h->featjobs.cap + h->feats.cap + h->mlpout.cap + h->chkjobs.cap +
                    h->chkratio.cap;
  for (auto& H : h->heights) {
    for (DevBuf* b : {&H.mr, &H.tbuf, &H.permbuf, &H.rankbuf, &H.refbuf, &H.clists, &H.idjobs, &H.slices,
                      &H.skmeta, &H.D, &H.piv, &H.rxpiv, &H.info, &H.X, &H.RX, &H.At, &H.qbuf, &H.flists,
                      &H.lujobs, &H.cjobs, &H.G, &H.FT, &H.TMP, &H.slists})
      bytes += (long long)b->cap;
  }
  h->st.device_bytes = bytes;
  h->st.ms_lu = 0;
  *out = h->st;
  return SYMHSS_OK;
}

int symhss_problem_ranks(symhss_t h, int problem, int level, int* out) {
  if (!h || !out || problem < 0 || problem >= (int)h->probs.size()) return SYMHSS_ERR_INVALID;
  const Problem& P = h->probs[problem];
  if (level < 1 || level > P.depth) return SYMHSS_ERR_INVALID;
  if (!h->compressed) return SYMHSS_ERR_STATE;
  const auto& bxs = P.levels[level];
  for (size_t b = 0; b < bxs.size(); ++b) {
    out[2 * b] = bxs[b].rank[0];
    out[2 * b + 1] = bxs[b].rank[1];
  }
  return SYMHSS_OK;
}

int symhss_level_ranks(symhss_t h, int level, int* out) { return symhss_problem_ranks(h, 0, level, out); }

static bool tuning_ok(const symhss_tuning* t) {
  auto in = [](int v, std::initializer_list<int> l) {
    for (int x : l)
      if (v == x) return true;
    return false;
  };
  return in(t->lu_lookahead, {0, 1}) && in(t->lu_panel_threads, {256, 512, 1024}) &&
         in(t->tile_loop_chunk, {0, 8, 16, 32}) && in(t->id_cluster_max, {1, 2, 4, 8, 16}) &&
         in(t->lu_panel_cluster, {1, 2, 4, 8, 16}) && in(t->lu_tc, {0, 1, 2}) && in(t->lu_outer, {0, 16, 32, 64});
}

int symhss_get_tuning(symhss_t h, symhss_tuning* out) {
  if (!h || !out) return SYMHSS_ERR_INVALID;
  *out = h->tune;
  return SYMHSS_OK;
}

int symhss_set_tuning(symhss_t h, const symhss_tuning* t) {
  if (!h || !t || !tuning_ok(t)) return SYMHSS_ERR_INVALID;
  h->tune = *t;
  return SYMHSS_OK;
}

int symhss_autotune(symhss_t h, int reps, symhss_tuning* out, void* stream) {
  BudgetScope budget_scope(h ? &h->budget : nullptr);
  if (!h || reps < 1 || reps > 100) return SYMHSS_ERR_INVALID;
  symhss_tuning best = h->tune;
  // min over reps of one kernel class's device time in compress
  auto time_compress = [&](int cls, double* ms) -> int {
    double m = 1e300;
    for (int r = 0; r < reps; ++r) {
      int rc = symhss_compress(h, stream);
      if (rc) return rc;
      m = std::min(m, h->st.kernel_ms[cls]);
    }
    *ms = m;
    return SYMHSS_OK;
  };
  double bms = 1e300, ms = 0;
  for (int v : {0, 8, 16, 32}) {
    h->tune = best;
    h->tune.tile_loop_chunk = v;
    int rc = time_compress(SYMHSS_K_TILES, &ms);
    if (rc) return rc;
    if (ms < bms) { bms = ms; best.tile_loop_chunk = v; }
  }
  bms = 1e300;
  for (int v : {1, 2, 4, 8, 16}) {
    h->tune = best;
    h->tune.id_cluster_max = v;
    int rc = time_compress(SYMHSS_K_ID, &ms);
    if (rc) return rc;
    if (ms < bms) { bms = ms; best.id_cluster_max = v; }
  }
  h->tune = best;
  int rc = symhss_compress(h, stream);
  if (rc) return rc;
  // the factorisation's arithmetic path and its block width: block LU and solve classes together
  bms = 1e300;
  const int paths[7][2] = {{2, 64}, {2, 32}, {2, 16}, {1, 64}, {1, 32}, {1, 16}, {0, 64}};
  for (const auto& pv : paths) {
    h->tune = best;
    h->tune.lu_tc = pv[0];
    h->tune.lu_outer = pv[1];
    double m = 1e300;
    for (int r = 0; r < reps; ++r) {
      const double b0 = h->st.kernel_ms[SYMHSS_K_GETRF] + h->st.kernel_ms[SYMHSS_K_GETRS];
      rc = symhss_factor(h, stream);
      if (rc) return rc;
      m = std::min(m, h->st.kernel_ms[SYMHSS_K_GETRF] + h->st.kernel_ms[SYMHSS_K_GETRS] - b0);
    }
    if (m < bms) { bms = m; best.lu_tc = pv[0]; best.lu_outer = pv[1]; }
  }
  bms = 1e300;
  for (int pt : {256, 512, 1024})
    for (int la : {0, 1}) {
      h->tune = best;
      h->tune.lu_panel_threads = pt;
      h->tune.lu_lookahead = la;
      double m = 1e300;
      for (int r = 0; r < reps; ++r) {
        const double before = h->st.kernel_ms[SYMHSS_K_GETRF];
        rc = symhss_factor(h, stream);
        if (rc) return rc;
        m = std::min(m, h->st.kernel_ms[SYMHSS_K_GETRF] - before);
      }
      if (m < bms) { bms = m; best.lu_panel_threads = pt; best.lu_lookahead = la; }
    }
  // panel cluster and look-ahead together: a cluster panel is short enough to hide behind the
  // trailing update on the side stream, a one-block panel is not
  bms = 1e300;
  for (int pcv : {1, 2, 4, 8, 16})
    for (int la : {0, 1}) {
      h->tune = best;
      h->tune.lu_panel_cluster = pcv;
      h->tune.lu_lookahead = la;
      double m = 1e300;
      for (int r = 0; r < reps; ++r) {
        const double before = h->st.kernel_ms[SYMHSS_K_GETRF];
        rc = symhss_factor(h, stream);
        if (rc) return rc;
        m = std::min(m, h->st.kernel_ms[SYMHSS_K_GETRF] - before);
      }
      if (m < bms) { bms = m; best.lu_panel_cluster = pcv; best.lu_lookahead = la; }
    }
  h->tune = best;
  rc = symhss_factor(h, stream);
  if (rc) return rc;
  if (out) *out = best;
  return SYMHSS_OK;
}

int symhss_set_rank_limit(symhss_t h, int max_rank) {
  if (!h) return SYMHSS_ERR_INVALID;
  h->rank_limit = max_rank > 0 ? max_rank : 0;
  return SYMHSS_OK;
}

int symhss_set_memory_limit(symhss_t h, long long bytes) {
  if (!h) return SYMHSS_ERR_INVALID;
  h->budget.limit = bytes > 0 ? bytes : 0;
  return SYMHSS_OK;
}

int symhss_set_proposer(symhss_t h, symhss_mlp_t net, double margin) {
  if (!h || !(margin >= 1.0) || !std::isfinite(margin)) return SYMHSS_ERR_INVALID;
  h->mlp = net;
  h->prop_margin = margin;
  return SYMHSS_OK;
}

int symhss_training_data(symhss_t h, int* count, float* x, float* y_rank, float* y_skel, float* mask, int* meta,
                         double* geo, void* stream) {
  if (!h || !count) return SYMHSS_ERR_INVALID;
  if (!h->compressed) return SYMHSS_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    std::vector<BoxRef> all, refs;
    for (int t = 0; t < h->maxdepth; ++t) {
      height_boxes(h, t, false, refs);
      all.insert(all.end(), refs.begin(), refs.end());
    }
    const int total = (int)all.size();
    const bool want = x || y_rank || y_skel || mask || meta || geo;
    if (!want) {
      *count = total;
      return SYMHSS_OK;
    }
    if (*count < total) return SYMHSS_ERR_INVALID;
    *count = total;
    if (total == 0) return SYMHSS_OK;
    std::vector<FeatJob> fj(total);
    for (int i = 0; i < total; ++i) {
      const BoxRef& rf = all[i];
      const HBox& bx = *rf.bx;
      const Problem& P = h->probs[rf.p];
      const int t = P.depth - rf.l;
      FeatJob f;
      f.cx = bx.cx; f.cy = bx.cy; f.rho = bx.rho; f.k0 = P.prm.k0; f.k1 = P.prm.k1; f.tol = h->prm.tol;
      f.begin = bx.begin; f.len = bx.end - bx.begin; f.height = t;
      f.n0 = (int)bx.act[0].size(); f.n1 = (int)bx.act[1].size(); f.m_near = bx.m_near; f.nproxy = bx.P;
      f.pad_ = 0;
      fj[i] = f;
      const int L = bx.end - bx.begin;
      for (int hh = 0; hh < 2; ++hh) {
        if (y_rank) y_rank[2 * i + hh] = (float)(std::log2(1.0 + bx.rank[hh]) / 8.0);
        if (y_skel || mask) {
          double cnt[32] = {}, hit[32] = {};
          std::vector<char> sk(L, 0);
          for (int j = 0; j < bx.rank[hh]; ++j) sk[bx.act[hh][bx.perm[hh][j]] - bx.begin] = 1;
          for (int q : bx.act[hh]) {
            const int j = (int)(((long long)(q - bx.begin) * 32) / L);
            cnt[j] += 1;
            hit[j] += sk[q - bx.begin];
          }
          for (int j = 0; j < 32; ++j) {
            if (y_skel) y_skel[(size_t)64 * i + 32 * hh + j] = cnt[j] > 0 ? (float)(hit[j] / cnt[j]) : 0.0f;
            if (mask) mask[(size_t)64 * i + 32 * hh + j] = cnt[j] > 0 ? 1.0f : 0.0f;
          }
        }
      }
      if (meta) {
        int* mt = meta + (size_t)10 * i;
        mt[0] = rf.p; mt[1] = rf.l; mt[2] = t; mt[3] = bx.begin - P.node0; mt[4] = L;
        mt[5] = f.n0; mt[6] = f.n1; mt[7] = bx.m_near; mt[8] = bx.P; mt[9] = 0;
      }
      if (geo) { geo[3 * i] = bx.cx; geo[3 * i + 1] = bx.cy; geo[3 * i + 2] = bx.rho; }
    }
    if (x) {
      Packer fp;
      fp.add(fj);
      CK(fp.upload(h->featjobs, s));
      CK(h->feats.ensure((size_t)total * kMlpWidth * sizeof(float)));
      CK(launch_box_features(table_of(h), h->featjobs.as<FeatJob>(), total, h->feats.as<float>(), s));
      CK(cudaMemcpyAsync(x, h->feats.p, (size_t)total * kMlpWidth * sizeof(float), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    return SYMHSS_OK;
  } catch (const std::bad_alloc&) {
    return SYMHSS_ERR_NOMEM;
  }
}

int symhss_destroy(symhss_t h) {
  if (!h) return SYMHSS_OK;
  if (h->cstream) cudaStreamDestroy(h->cstream);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->evpool) cudaEventDestroy(e);
  delete h;
  return SYMHSS_OK;
}

}  // extern "C"
