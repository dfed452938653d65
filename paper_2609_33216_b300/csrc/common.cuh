// Shared device helpers of the symhss library: complex128 arithmetic on double2,
// block reductions, job descriptors and launcher declarations.
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <stdint.h>

#include "../../include/symhss.h"

namespace symhss {

// ---- complex128 on double2 (x = re, y = im) ---------------------------------

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
// acc += conj(a) * b, four fused multiply-adds
__device__ __forceinline__ double2 cconjfma(double2 a, double2 b, double2 acc) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
// acc + |a|^2, two fused multiply-adds
__device__ __forceinline__ double cabs2_acc(double2 a, double acc) { return fma(a.x, a.x, fma(a.y, a.y, acc)); }
// acc += a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// acc -= a * b
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 acc) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ double2 cinv(double2 a) {
  // 1/a with scaling against overflow (Smith's method)
  if (fabs(a.x) >= fabs(a.y)) {
    double r = a.y / a.x, d = a.x + a.y * r;
    return make_double2(1.0 / d, -r / d);
  } else {
    double r = a.x / a.y, d = a.y + a.x * r;
    return make_double2(r / d, -1.0 / d);
  }
}

// ---- complex64 on float2 (the mixed-precision factorisation) ----------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ float cabs1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
__device__ __forceinline__ float2 cinv(float2 a) {
  if (fabsf(a.x) >= fabsf(a.y)) {
    float r = a.y / a.x, d = a.x + a.y * r;
    return make_float2(1.0f / d, -r / d);
  } else {
    float r = a.x / a.y, d = a.y + a.x * r;
    return make_float2(r / d, -1.0f / d);
  }
}
// 1 / d for d > 0 with a biased exponent in [27, 2019]: Newton's iteration for the reciprocal,
// r <- r + r (1 - d r), whose relative error squares at each step, taken twice from the
// hardware's approximate reciprocal (rcp.approx.ftz.f64); the result is within about one unit
// in the last place of the rounded quotient 1.0 / d.  Four fused multiply-adds on the FP64
// pipe, against the longer sequence of a full division (this GPU issues FP64 instructions
// slowly, and the pivot's reciprocal is on the LU panel's serial chain).
__device__ __forceinline__ double recip_newton(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}
// Reciprocal of an LU pivot on a serial dependency chain: conj(a) / |a|^2 with the reciprocal
// of |a|^2 by recip_newton; Smith's scaled form is kept for |a|^2 outside [2^-996, 2^997)
// (tested on the exponent bits), where the plain form would overflow or underflow.
__device__ __forceinline__ double2 cinv_pivot(double2 a) {
  const double s2 = fma(a.x, a.x, a.y * a.y);
  const int ex = (int)((__double_as_longlong(s2) >> 52) & 0x7FF);
  if (ex < 27 || ex > 2019) return cinv(a);
  const double r = recip_newton(s2);
  return make_double2(a.x * r, -a.y * r);
}
__device__ __forceinline__ float2 cinv_pivot(float2 a) {
  const float s2 = fmaf(a.x, a.x, a.y * a.y);
  if (!(s2 > 1e-36f && s2 < 1e36f)) return cinv(a);
  const float r = 1.0f / s2;
  return make_float2(a.x * r, -a.y * r);
}
// complex constant / conversion in the element type CT (double2 or float2)
template <typename CT> __device__ __forceinline__ CT make_c(double re, double im);
template <> __device__ __forceinline__ double2 make_c<double2>(double re, double im) { return make_double2(re, im); }
template <> __device__ __forceinline__ float2 make_c<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <typename CT> __device__ __forceinline__ CT to_c(double2 v) { return make_c<CT>(v.x, v.y); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_csum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
// argmax over (value, index) with ties to the lowest index
__device__ __forceinline__ void warp_argmax(double& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
}

// Pivot-search keys: |re| + |im| >= 0 by its IEEE bit pattern, whose integer order is the
// order of the values for non-negative numbers (NaN maps below every number, so it is never
// picked).  Comparing keys keeps the pivot search on the integer pipes, which matters where
// FP64 issues at a small fraction of the FP32 rate.
__device__ __forceinline__ long long pivot_key(double v) {
  const long long k = __double_as_longlong(v);
  return k > 0x7ff0000000000000LL ? -1LL : k;
}
__device__ __forceinline__ long long pivot_key(float v) {
  const int k = __float_as_int(v);
  return k > 0x7f800000 ? -1LL : (long long)k;
}
// argmax over (key, index) with ties to the lowest index
__device__ __forceinline__ void warp_argmax_key(long long& k, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, k, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ok > k || (ok == k && oi < i)) { k = ok; i = oi; }
  }
}
// the same, carrying a payload x with the winning (k, i); every lane ends with the result
__device__ __forceinline__ void warp_argmax_key(long long& k, int& i, int& x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, k, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    const int ox = __shfl_xor_sync(0xffffffffu, x, o);
    if (ok > k || (ok == k && oi < i)) { k = ok; i = oi; x = ox; }
  }
}
// the same result (all lanes) through warp reductions instead of five shuffle rounds: the
// largest key as two 32-bit maxima (high word, then the low word among the lanes holding it;
// key + 1 so that "no candidate" = -1 maps to 0), then the lowest index among the lanes
// holding that key, then the payload of the lane holding both
__device__ __forceinline__ void warp_argmax_key_redux(long long& k, int& i, int& x) {
  const unsigned full = 0xffffffffu;
  const unsigned long long u = (unsigned long long)(k + 1);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned mh = __reduce_max_sync(full, hi);
  const unsigned ml = __reduce_max_sync(full, hi == mh ? lo : 0u);
  const bool top = hi == mh && lo == ml;
  const int mi = __reduce_min_sync(full, top ? i : 0x7fffffff);
  const unsigned win = __ballot_sync(full, top && i == mi);
  x = __shfl_sync(full, x, __ffs(win) - 1);
  k = (long long)(((unsigned long long)mh << 32) | ml) - 1;
  i = mi;
}

// Programmatic dependent launch: a kernel launched with it may be scheduled while the kernel
// before it in the stream is still running.  Every thread waits here for that kernel (its
// completion and its memory) before the first global-memory access and before any exit, and
// then lets the next such kernel be scheduled.  Without a programmatic launch both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// A kernel launch, as a programmatic dependent of the kernel before it on the stream when
// `chained` (then the kernel must begin with pdl_enter), else a plain launch.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(bool chained, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                  cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// process-wide count of kernels this library has launched (diagnostics)
void count_launches(long long n);

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, cached per
// device; 148 on a B300 if the query fails).  Used to size grids in multiples of the SM count.
int device_sm_count();

// device status bits (OR-ed into a device word the host reads at sync points)
enum : int {
  ST_BAD_INDEX = 1,
  ST_RANK_OVERFLOW = 2,
  ST_SINGULAR = 4,
  ST_SMEM = 8,
  ST_TIMEOUT = 16,
};

// ---- tile generator ---------------------------------------------------------

// Point table (structure of arrays).  id >= 0 marks a curve node.  hs: the node's
// parametrisation-speed term of the hypersingular diagonal (speed_terms; NULL reads as 0).
struct PointTable {
  const double *x, *y, *nx, *ny, *w, *kappa;
  const int* id;
  const double* hs;
};

// Speed term of the one-point corrected hypersingular diagonal for one closed curve with
// trapezoidal weights w[0..n) (see symhss_speed_terms in symhss.h): host code.
void speed_terms(const double* w, int n, double* out);

// Physical constants of one system.
// Per-problem constants of the tile generator.  The blocks are combinations of the layer
// kernels of the two wavenumbers:
//   A11 = -w (cs0 S_k0 - cs1 S_k1)      A12 = w (cd0 D_k0 - cd1 D_k1) - ft
//   A21 = w (cd0 D*_k0 - cd1 D*_k1) + ft  A22 = -w (cn0 N_k0 - cn1 N_k1)
// Muller-like (Eq. 15): cs = (eps0^2, eps1^2), cd = (eps0, eps1), cn = (1, 1), ft = (eps0 + eps1)/2;
// PMCHWT (Eq. symmetric_pmchwt): cs = (eps0, -eps1), cd = (1, -1), cn = (1/eps0, -1/eps1), ft = 0.
struct KernelParams {
  double k0, k1, eps0, eps1;
  double cs0, cs1, cd0, cd1, cn0, cn1;
  double half_ft;      // free term (eps0 + eps1) / 2, or 0
  double lhk0, lhk1;   // log(k0 / 2), log(k1 / 2)
  double ik0, ik1;     // 1 / k0, 1 / k1
  int form;            // SYMHSS_MULLER or SYMHSS_PMCHWT
  int pad_;
};

inline KernelParams make_kernel_params(const symhss_params& p) {
  KernelParams k;
  k.k0 = p.k0; k.k1 = p.k1; k.eps0 = p.eps0; k.eps1 = p.eps1;
  k.form = p.formulation;
  k.pad_ = 0;
  if (p.formulation == SYMHSS_BM) {  // only the layer kernels are combined in the tile kernel's BM branch
    k.cs0 = p.eps0; k.cs1 = p.eps1; k.cd0 = 1.0; k.cd1 = 1.0; k.cn0 = 1.0 / p.k0; k.cn1 = 0.0;
    k.half_ft = 0.5;
  } else if (p.formulation == SYMHSS_PMCHWT) {
    k.cs0 = p.eps0; k.cs1 = -p.eps1; k.cd0 = 1.0; k.cd1 = -1.0; k.cn0 = 1.0 / p.eps0; k.cn1 = -1.0 / p.eps1;
    k.half_ft = 0.0;
  } else {
    k.cs0 = p.eps0 * p.eps0; k.cs1 = p.eps1 * p.eps1; k.cd0 = p.eps0; k.cd1 = p.eps1; k.cn0 = 1.0; k.cn1 = 1.0;
    k.half_ft = 0.5 * (p.eps0 + p.eps1);
  }
  k.lhk0 = std::log(0.5 * p.k0);
  k.lhk1 = std::log(0.5 * p.k1);
  k.ik0 = 1.0 / p.k0;
  k.ik1 = 1.0 / p.k1;
  return k;
}

// A tile: "thread points" (one per thread) x "loop points" (staged in shared
// memory).  Each point carries two output slots (-1 = absent): for observation
// points the rows of equation 1 and 2, for source points the columns of the
// flux and trace unknowns.  Element (thread slot s, loop slot t) is written to
// out[out_off + s + t * ld].
struct TileJob {
  int tp_off, n_tp;        // thread points: [tp_off, tp_off + n_tp) of the thread lists
  int lp_off, n_lp;        // loop points
  long long out_off;
  int ld;
  int flags;               // TILE_SRC_IS_THREAD: thread points are sources (transposed output)
                           // TILE_UNSCALED: the baseline system of Sec. 6
  int prm;                 // index of this job's physical constants in TileLaunch::kps
  int pad_;
};
// TILE_SYM_DIAG: a symmetric diagonal block whose thread points are its loop points (same
// list): only pairs j >= i are evaluated and each j > i is written twice, once transposed
// (the symmetric system's matrix is exactly symmetric off the node diagonal)
enum : int { TILE_SRC_IS_THREAD = 1, TILE_UNSCALED = 2, TILE_SYM_DIAG = 4 };

struct TileChunk { int job, t0, l0, ln; };  // ln: loop points of this chunk (<= TILE_L)

struct TileLaunch {
  PointTable tpts, lpts;   // tables the thread / loop point indices refer to
  const int *tp_pt, *tp_s0, *tp_s1;
  const int *lp_pt, *lp_s0, *lp_s1;
  const TileJob* jobs;
  const TileChunk* chunks;
  int nchunks;
  double2* out;
  int* status;
  const KernelParams* kps;  // device array, one entry per problem
};

constexpr int TILE_T = 128;   // thread points per chunk (= threads per block)
constexpr int TILE_L = 32;    // loop points per chunk

cudaError_t launch_tiles(const TileLaunch& a, cudaStream_t s);
cudaError_t launch_hankel(const double* x, int n, double2* out, cudaStream_t s);
// out[i] = the LU panels' pivot reciprocal (cinv_pivot) of a[i], n complex128 values
cudaError_t launch_pivot_reciprocal(const double2* a, int n, double2* out, cudaStream_t s);

// ---- column ID (pivoted QR) ---------------------------------------------------

struct IdJob {
  long long m_off;   // M at mats + m_off (column-major, leading dim ld)
  int m, n, ld;
  int start;         // first QR step (0 = fresh; > 0 continues a previous run)
  int fixed;         // < 0: tolerance stop; else stop after `fixed` steps
  long long t_off;   // T output at tbuf + t_off (leading dim = rank)
  long long perm_off;
  int out_idx;       // rank[out_idx], ref[out_idx]
};

struct IdLaunch {
  int cluster_max = 16;  // largest cluster per ID
  double2* mats;
  double2* tbuf;
  int* perm;
  int* rank;
  double* ref;       // |R_00| of each job (kept for continuation runs)
  const IdJob* jobs;
  int njobs;
  double tol;
  int* status;
  int max_m, max_n;
};
cudaError_t launch_cpqr(const IdLaunch& a, cudaStream_t s);
int cpqr_cluster_size(int njobs, int max_n);

// Interpolation residual of an ID on a set of rows (the check that accepts a sketched ID,
// run on held-out sketch rows): ratio[out] = max over non-skeleton columns c of
// ||M[:, c] - M[:, J] T[:, c]|| divided by the largest column norm of M (J = perm[0 .. rank),
// T = R11^{-1} R12 with leading dimension rank).
// One ID checked on its proxy matrix M (m x n at m_off, leading dimension ld): its skeleton
// columns go to g + g1_off (m x r), the others to g + g2_off (m x (n - r)), both with leading
// dimension m (idcheck.cu).
struct GatherJob {
  long long m_off;
  int m, n, ld, r;
  long long perm_off;
  long long g1_off, g2_off;
};
cudaError_t launch_gather_cols(const double2* mats, const int* perm, const GatherJob* jobs, const int2* work,
                               int nwork, double2* g, cudaStream_t s);
cudaError_t launch_residual_ratio(const double2* mats, const double2* g, const GatherJob* jobs, const int* outs,
                                  int njobs, double* ratio, cudaStream_t s);

struct CheckJob {
  long long m_off;   // M at mats + m_off (column-major, leading dim ld)
  int m, n, ld;
  int rank_idx;      // rank[rank_idx]
  long long t_off;   // T at tbuf + t_off
  long long perm_off;
  int out;           // ratio[out]
  int pad_;
};
cudaError_t launch_id_check(const double2* mats, const double2* tbuf, const int* perm, const int* rank,
                            const CheckJob* jobs, int njobs, double* ratio, cudaStream_t s);

// ---- learned rank / skeleton proposer --------------------------------------------------
// A 128-128-128 ReLU MLP with FP16 weights and FP32 accumulation (parameters packed as
// [W1 (row-major out x in), b1, W2, b2, W3, b3]); input: 128 box features, output 0 / 1:
// log2(1 + rank) / 8 of the flux / trace half, 2..33 / 34..65: skeleton logits.
constexpr int kMlpWidth = 128;
constexpr int kMlpOutUsed = 66;
constexpr int kMlpLayerParams = kMlpWidth * kMlpWidth + kMlpWidth;
constexpr int kMlpParams = 3 * kMlpLayerParams;

// Features of one box (see the feature definition in mlp.cu).
struct FeatJob {
  double cx, cy, rho, k0, k1, tol;
  int begin, len, height, n0, n1, m_near, nproxy, pad_;
};
cudaError_t launch_box_features(const PointTable& t, const FeatJob* jobs, int njobs, float* out, cudaStream_t s);
cudaError_t mlp_forward(symhss_mlp_s* net, const float* x, int batch, float* out, cudaStream_t s);

// ---- randomized sketch Y = Omega M on the tensor cores --------------------------------

struct SketchJob {
  long long m_off;     // M at mats + m_off (m x n complex, leading dim ld)
  int m, n, ld;
  int mpad, n2pad;     // m rounded up to 64, 2n rounded up to 32
  int s;               // rows of Y (<= 128 * number of row tiles)
  long long y_off;     // Y at y + y_off (s x n complex, leading dim ldy)
  int ldy;
  long long slice_off; // bytes into the slice buffer
  long long exp_off;   // ints into the exponent buffer (2n entries)
  long long stream_id; // counter-stream index of this job's Omega
};
struct SketchColWork { int job, col; };
struct SketchTile { int job, cb, mtile; };
struct SketchLaunch {
  const double2* mats;
  uint8_t* slices;
  int* exps;
  double2* y;
  const SketchJob* jobs;
  const SketchColWork* colwork;
  int ncolwork;
  const SketchTile* tiles;
  int ntiles;
  uint64_t seed;
  int* status;
  long long wait_ns;   // time limit of each pipeline wait (the drain after a timeout keeps the default)
};
cudaError_t launch_sketch(const SketchLaunch& a, cudaStream_t s);
// Time limit of the sketch kernel's pipeline waits for launches made from now on (ns; <= 0
// restores the default): a test hook for the timeout path.
void set_sketch_wait_ns(long long ns);
size_t sketch_slice_bytes(int mpad, int n2pad);
int sketch_mpad(int m);
int sketch_n2pad(int n);
uint64_t sketch_host_splitmix64(uint64_t x);

// ---- batched LU and solves -----------------------------------------------------

struct LuJob {
  long long a_off;  // matrix at base + a_off
  int n, ld;
  long long piv_off;
  int info_idx;
};
struct LuLaunch {
  double2* base;
  int* piv;
  int* info;
  const LuJob* jobs;
  int njobs;
  int max_n;
  int* status;
  float2* base32 = nullptr;  // non-null: factor these complex64 matrices instead of `base`
  int lookahead = 1;       // depth-1 look-ahead on a side stream
  int panel_threads = 1024;  // largest panel block
  int panel_cluster = 1;     // largest cluster for the panels of few large matrices (1: one block)
  int tc = 2;                // FP64: column blocks with tensor-core updates (1: always, 2: for
                             // launches of at least 32 matrices, 0: never)
  int outer = 64;            // their width: 16 (a tensor-core update after every panel), 32 or 64
  unsigned char* zimg = nullptr;  // tensor-core product scratch, zgemm_lu_img_bytes(njobs, max_n)
  long long zimg_bytes = 0;       // bytes (too few: the FP64-pipe path)
  int* perm = nullptr;            // optional: the row permutation of every matrix (at piv_off),
                                  // kept current by the interchange kernel (x = P b: x[i] = b[perm[i]])
};
cudaError_t launch_getrf(const LuLaunch& a, cudaStream_t s);

struct RsJob {
  long long a_off; int n, lda; long long piv_off;
  long long b_off; int ldb; int nrhs;
};
struct RsLaunch {
  const double2* abase;
  const int* piv;
  double2* bbase;
  const float2* abase32 = nullptr;  // non-null: complex64 factors and right-hand sides
  float2* bbase32 = nullptr;
  const RsJob* jobs;
  int njobs;
  int max_rhs;
  int max_n;
  int* status = nullptr;  // device status word; needed (with tc) by the tensor-core path
  int tc = 2;             // FP64, > 4 right-hand sides, n > 64: blocked solve with tensor-core updates
                          // (1: always, 2: for launches of at least 32 matrices, 0: never)
  unsigned char* zimg = nullptr;  // tensor-core product scratch, zgemm_rs_img_bytes(njobs, max_n, max_rhs)
  long long zimg_bytes = 0;       // bytes (too few: the unblocked FP64 solve)
  const int* perm = nullptr;      // optional: the LU's row permutations (LuLaunch::perm); else
                                  // every solve composes them from piv
  int blk = 64;                   // row block of the blocked tensor-core solve: 16, 32 or 64
  double2* dinv = nullptr;        // optional scratch, getrs_dinv_bytes(njobs, max_n): the blocked
  long long dinv_bytes = 0;       // solve with 64-row blocks then solves its diagonal blocks
                                  // through their inverses on the tensor cores
};
cudaError_t launch_getrs(const RsLaunch& a, cudaStream_t s);
// bytes of RsLaunch::dinv: two 64 x 64 complex128 blocks (the inverses of L's unit-lower and U's
// upper diagonal block) per 64-row block of every matrix
long long getrs_dinv_bytes(int njobs, int max_n);
// scratch of the tensor-core products of a blocked LU / blocked solve launch
long long zgemm_lu_img_bytes(int njobs, int max_n);
long long zgemm_rs_img_bytes(int njobs, int max_n, int max_rhs);

// ---- complex FP64 GEMM on the tensor cores (zgemm_tc.cu) ---------------------------

enum : int { ZGEMM_SET = 0, ZGEMM_SUB = 1, ZGEMM_ADD = 2 };  // C = AB, C -= AB, C += AB
struct ZgemmJob {
  long long a_off, b_off, c_off;  // complex offsets of A (m x k), B (k x n), C (m x n)
  int m, n, k;                    // k <= zgemm_tc_max_k()
  int lda, ldb, ldc;
};
struct ZgemmTile { int job, mt, nt; };  // row tile mt (128 rows), column tile nt (32 columns)
// Jobs derived on the device from the factorisation's job arrays (block J = 64-aligned row):
enum : int {
  ZGEMM_JOBS = 0,      // explicit ZgemmJob / ZgemmTile arrays
  ZGEMM_LU_UPDATE = 1,  // LuJob: A[J+W:n, J+W:n] -= A[J+W:n, J:J+W] A[J:J+W, J+W:n], W = block_w
  ZGEMM_RS_FWD = 2,     // RsJob: X[J+W:n, :] -= L[J+W:n, J:J+W] X[J:J+W, :]
  ZGEMM_RS_BWD = 3,     // RsJob: X[0:J, :] -= U[0:J, J:J+W] X[J:J+W, :]
  ZGEMM_RS_FWD_DIAG = 4,  // RsJob: X[J:J+W, :] = inv(L[J:J+W, J:J+W]) X[J:J+W, :] (A: the inverse scratch)
  ZGEMM_RS_BWD_DIAG = 5,  // RsJob: X[J:J+W, :] = inv(U[J:J+W, J:J+W]) X[J:J+W, :] (A: the inverse scratch)
};
struct ZgemmLaunch {
  const double2* A;
  const double2* B;
  double2* C;
  const ZgemmJob* jobs;
  const ZgemmTile* tiles;
  int ntiles;          // grid size (derived jobs: njobs x mtiles x ntiles, idle tiles exit)
  int mode;            // ZGEMM_SET / ZGEMM_SUB / ZGEMM_ADD
  int* status;         // ST_TIMEOUT is OR-ed in when a bounded wait expires
  long long wait_ns;   // set by launch_zgemm_tc
  int derive = ZGEMM_JOBS;
  const LuJob* lu_jobs = nullptr;
  const RsJob* rs_jobs = nullptr;
  int block_j = 0;     // J of the derived jobs
  int block_w = 64;    // W: width of the column block J .. J + W of the derived jobs
  int inv_nb = 0;      // RS_*_DIAG: 64-row blocks per matrix in the inverse scratch (A)
  int mtiles = 0, ntiles_c = 0;  // row / column blocks per job (explicit jobs: the largest)
  int njobs = 0;                   // jobs of the launch
  int inline_slice = 0;            // every job has k <= 16: each tile slices its own operands
                                   // (no slicing launch, no images; img may be null)
  int chained = 0;                 // the first kernel of the product (the slicing kernel, or
                                   // with inline_slice the product kernel) is a programmatic
                                   // dependent launch of the kernel before it in the stream
  unsigned char* img = nullptr;    // scratch for the slice images (16-byte aligned),
  long long img_bytes = 0;         // at least zgemm_img_bytes(njobs, mtiles, ntiles_c)
  int probe_timeout = 0;           // set by launch_zgemm_tc (test hook, see set_zgemm_timeout_probe)
};
cudaError_t launch_zgemm_tc(const ZgemmLaunch& a, cudaStream_t s);
void set_zgemm_wait_ns(long long ns);
// test hook: while on, the last MMA wait of every product launch targets a phase that no
// commit completes, so it expires after the wait limit (the kernel then drains its MMAs)
void set_zgemm_timeout_probe(int on);
int zgemm_tc_tile_rows();
int zgemm_tc_tile_cols();
int zgemm_tc_max_k();
// scratch bytes of a launch of njobs jobs with mtiles x ntiles blocks each (or of m x n jobs)
long long zgemm_img_bytes(int njobs, int mtiles, int ntiles);
long long zgemm_img_bytes_for(int njobs, int max_m, int max_n);


// ---- factor / solve helpers ------------------------------------------------------

// Interpolation basis of one box in its diagonal-block ordering (Sec. 4.1): for
// part h (flux / trace), q[c] (c < n_h) is the diagonal-block position of the c-th
// pivoted active unknown; the first r_h are the skeleton.  T is r_h x (n_h - r_h)
// with leading dimension r_h, and R^h = [I T] Pi^T.
struct BasisPart {
  long long q_off;   // into the int buffer
  long long t_off;   // into the T buffer
  int n, r;
  int col0;          // first row/column of this part among the box's k = r_0 + r_1
};
struct BasisJob {
  BasisPart part[2];
  int size;          // diagonal-block order
  int k;             // r_0 + r_1
  long long in_off;  // input (size x ncols, leading dim ld_in)   [apply_r]
  int ld_in;
  long long out_off; // output: dense basis (size x k, leading dim size) [basis_dense]
  int ld_out;        //         or R * input (k x ncols, leading dim ld_out) [apply_r]
  int ncols;
};
struct BasisLaunch {
  const int* q;
  const double2* T;
  const double2* in;
  double2* out;
  const float2* in32 = nullptr;  // non-null out32: complex64 in / out (T stays complex128)
  float2* out32 = nullptr;
  const BasisJob* jobs;
  int njobs;
  int max_cols;
};
// out = dense R^T (equivalently L for a row basis): 1 at skeleton rows, T^T below
cudaError_t launch_basis_dense(const BasisLaunch& a, cudaStream_t s);
// out = R * in
cudaError_t launch_apply_r(const BasisLaunch& a, cudaStream_t s);

// C = alpha * A * B + beta * C for batches of small complex matrices (alpha, beta real)
struct GemmJob {
  long long a_off, b_off, c_off;
  int lda, ldb, ldc;
  int m, n, k;
  double alpha, beta;
};
struct GemmLaunch {
  const double2* A;
  const double2* B;
  double2* C;
  const GemmJob* jobs;
  int njobs;
  int max_m = 0;  // largest m and n over the jobs (0: unknown, the tiled kernel runs)
  int max_n = 0;
};
cudaError_t launch_gemm(const GemmLaunch& a, cudaStream_t s);

// dst block (rows x cols, ldd) = src block (lds); identity fill when src_off < 0
// dst(i, j) = src(i, j) for a rows x cols block; trans != 0: dst(j, i) = src(i, j)
struct CopyJob { long long src_off, dst_off; int rows, cols, lds, ldd; int trans = 0; int pad_ = 0; };
cudaError_t launch_copy_blocks(const double2* src, double2* dst, const CopyJob* jobs, int njobs,
                               cudaStream_t s);
cudaError_t launch_copy_blocks32(const float2* src, float2* dst, const CopyJob* jobs, int njobs, cudaStream_t s);
// element-wise precision changes of n complex values
cudaError_t launch_narrow(const double2* src, float2* dst, long long n, cudaStream_t s);
cudaError_t launch_widen(const float2* src, double2* dst, long long n, cudaStream_t s);
// out += L * in: the transpose of apply_r (skeleton rows get in, the others T^T in)
cudaError_t launch_apply_l(const BasisLaunch& a, cudaStream_t s);
// y = a x + b y, elementwise over n complex values (a, b real)
cudaError_t launch_axpby(const double2* x, double2* y, long long n, double a, double b, cudaStream_t s);

// Leaf boxes are contiguous node ranges [begin, begin + len) of a problem with n
// nodes whose [eq1; eq2] block starts at `base` in the global vectors; the box
// vector holds [eq1 rows; eq2 rows] of the box (size 2 len) with nrhs columns.
struct LeafJob { long long off; long long base; int begin, len, n, pad_; };
cudaError_t launch_leaf_gather(const double2* f, long long ldf, double2* g, const LeafJob* jobs, int njobs,
                               int nrhs, cudaStream_t s);
cudaError_t launch_leaf_scatter(const double2* g, double2* x, long long ldx, const LeafJob* jobs,
                                int njobs, int nrhs, cudaStream_t s);

// Plane-wave right-hand side of problem jobs[j]: nodes [node0, node0 + n) of the
// point table, rows [vec0, vec0 + 2n) of rhs ([eq1; eq2]).
// rhs rows: [a1 u_in + b1 du_in/dnu ; a2 u_in + b2 du_in/dnu], times W for the row-scaled systems
struct WaveJob { int node0, n; long long vec0; double k0; double2 a1, b1, a2, b2; };
cudaError_t launch_plane_wave(const PointTable& t, const WaveJob* jobs, int njobs, int max_n, double angle,
                              int scaled, double2* rhs, cudaStream_t s);

}  // namespace symhss
