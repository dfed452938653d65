// Batched column interpolative decomposition by Householder QR with column
// pivoting (Sec. 4.1: the ID of each half of the proxy matrix M_R).
//
// Each matrix is factored by one thread-block cluster of C blocks (C = 1, 2, 4,
// 8 or 16, chosen per launch so that few large IDs still occupy many SMs).  Block
// `rank` of the cluster owns the columns j with j % C == rank; the matrix stays in
// global memory (L2-resident) and columns are never moved: the pivot order is
// kept in order[], and R(k, j) ends up at M(k, j).  Step k:
//   1. every block proposes its owned, not yet chosen column of largest remaining
//      norm; after a cluster barrier each block reads all proposals through
//      distributed shared memory and takes the largest (ties to the lowest index);
//   2. stop at the first pivot norm <= tol * (first pivot norm), or after `fixed`
//      steps;
//   3. the owner of the pivot column builds the reflector H = I - tau v v^H with
//      H x = alpha e_1 in its shared memory; after a second cluster barrier the
//      other blocks copy v and tau from it;
//   4. every block applies H to its remaining columns (one warp per column) and,
//      in the same pass, recomputes their remaining norms exactly.
// Afterwards T = R11^{-1} R12 is obtained by back substitution, one warp per
// redundant column.  perm = [chosen columns in pivot order, remaining columns in
// increasing index]; T's columns follow perm[r:].  A launch with start > 0 resumes
// a factorisation left by an earlier launch (used to raise a rank).
#include <cooperative_groups.h>

#include <type_traits>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace symhss {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct Cand { long long k; int i; };  // pivot key of the norm, column

__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s += red[w];
  return s;
}

__global__ void __launch_bounds__(kThreads) cpqr_cluster_kernel(const IdLaunch a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int job = blockIdx.x / C;
  const IdJob jb = a.jobs[job];
  double2* vbuf = reinterpret_cast<double2*>(smem_raw);           // max_m
  double* norms = reinterpret_cast<double*>(vbuf + a.max_m);      // max_n (owned entries)
  int* order = reinterpret_cast<int*>(norms + a.max_n);           // max_n
  int* done = order + a.max_n;                                     // max_n: 1 = chosen
  __shared__ double red[kWarps];
  __shared__ long long redk[kWarps];
  __shared__ int redi[kWarps];
  __shared__ Cand cand[2];
  __shared__ Cand s_pick;
  __shared__ double s_tau;
  __shared__ double2 s_alpha;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = jb.m, n = jb.n, ld = jb.ld;
  const bool bad = (m > a.max_m || n > a.max_n || m < 0 || n < 0 || jb.start < 0);
  if (bad) {  // uniform over the cluster: every block of the job returns here
    if (tid == 0 && rank == 0) { atomicOr(a.status, ST_BAD_INDEX); a.rank[jb.out_idx] = 0; }
    return;
  }
  double2* M = a.mats + jb.m_off;
  int* perm_out = a.perm + jb.perm_off;
  const int start = min(jb.start, min(m, n));
  for (int j = tid; j < n; j += kThreads) done[j] = 0;
  __syncthreads();
  for (int i = tid; i < start; i += kThreads) {
    const int q = perm_out[i];
    order[i] = q;
    if (q >= 0 && q < n) done[q] = 1;
  }
  __syncthreads();
  int kmax = min(m, n);
  if (jb.fixed >= 0) kmax = min(kmax, jb.fixed);
  int k = start;
  // remaining norms of owned columns over rows k..m-1
  for (int j = rank + C * warp; j < n; j += C * kWarps) {
    const double2* col = M + (long long)j * ld;
    double s = 0.0;
    for (int i = k + lane; i < m; i += 32) s += cabs2(col[i]);
    s = warp_sum(s);
    if (lane == 0) norms[j] = sqrt(s);
  }
  double ref = (start == 0) ? -1.0 : a.ref[jb.out_idx];
  __syncthreads();

  int par = 0;
  while (true) {
    // 1. local proposal (integer keys of the non-negative norms: same order, integer pipes)
    long long bk = -1;
    int bi = n;
    for (int j = rank + C * tid; j < n; j += C * kThreads) {
      if (done[j]) continue;
      const long long kj = pivot_key(norms[j]);
      if (kj > bk || (kj == bk && j < bi)) { bk = kj; bi = j; }
    }
    warp_argmax_key(bk, bi);
    if (lane == 0) { redk[warp] = bk; redi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      bk = lane < kWarps ? redk[lane] : -1;
      bi = lane < kWarps ? redi[lane] : n;
      warp_argmax_key(bk, bi);
      if (lane == 0) cand[par] = Cand{bk, bi};
    }
    cl.sync();
    // the C proposals are read in parallel (one lane each) and reduced with shuffles
    if (warp == 0) {
      long long ck = -1;
      int ci = n;
      if (lane < C) {
        const Cand cd = *cl.map_shared_rank(&cand[par], lane);
        ck = cd.k;
        ci = cd.i;
      }
      warp_argmax_key(ck, ci);
      if (lane == 0) s_pick = Cand{ck, ci};
    }
    __syncthreads();
    const double pv = s_pick.k < 0 ? -1.0 : __longlong_as_double(s_pick.k);
    const int p = s_pick.i;
    par ^= 1;
    if (ref < 0.0) ref = pv;
    // 2. stop (the same decision in every block of the cluster)
    if (k >= kmax || p >= n || pv <= 0.0 || (jb.fixed < 0 && pv <= a.tol * ref)) break;
    const int owner = p % C;
    // 3. reflector, built by the owner (every block takes part in the reduction so
    //    that no barrier sits in a branch)
    double s = 0.0;
    if (rank == owner) {
      const double2* cp = M + (long long)p * ld;
      for (int i = k + tid; i < m; i += kThreads) {
        const double2 x = cp[i];
        vbuf[i - k] = x;
        s += cabs2(x);
      }
    }
    const double sigma2 = block_sum(s, red);
    if (rank == owner && tid == 0) {
      const double sigma = sqrt(sigma2);
      const double2 x0 = vbuf[0];
      const double ax0 = sqrt(cabs2(x0));
      const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
      s_alpha = make_double2(-ph.x * sigma, -ph.y * sigma);
      vbuf[0] = make_double2(ph.x * (ax0 + sigma), ph.y * (ax0 + sigma));
      const double vn2 = 2.0 * sigma * (sigma + ax0);
      s_tau = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
    }
    cl.sync();
    if (rank != owner) {
      const double2* rv = cl.map_shared_rank(vbuf, owner);
      for (int i = tid; i < m - k; i += kThreads) vbuf[i] = rv[i];
      if (tid == 0) s_tau = *cl.map_shared_rank(&s_tau, owner);
    }
    if (tid == 0) { done[p] = 1; order[k] = p; }
    __syncthreads();
    const double tau = s_tau;
    // 4. apply to owned remaining columns, recompute their remaining norms: LPC lanes per
    //    column, 32 / LPC columns per warp (LPC = 8: each column segment is one 128-byte line,
    //    the lane sums take 3 shuffle levels instead of 5; LPC = 16 for tall matrices, m >= 128,
    //    where a block owns few columns: twice the warps share them, so the busiest
    //    sub-partition's FP64 pipe carries less of the step).  The choice depends on the
    //    launch's largest m only, so every cluster size gives the same sums.
    //    Every sum is a chain of fused multiply-adds (4 per element for v^H c, 2 for |c|^2):
    //    the FP64 pipe bounds this loop on this GPU, and separate products and additions
    //    would issue 13 FP64 instructions per element instead of 10.
    auto apply_cols = [&](auto lpc) {
      constexpr int LPC = decltype(lpc)::value, CPW = 32 / LPC;
      const int grp = lane / LPC, gl = lane % LPC;
      const int nown = (n - rank + C - 1) / C;  // owned columns: j = rank + C * t, t < nown
      for (int t0 = CPW * warp; t0 < nown; t0 += CPW * kWarps) {  // uniform per warp
        const int t = t0 + grp;
        const int j = rank + C * t;
        const bool act = t < nown && j < n && !done[j];
        double2* col = M + (long long)(act ? j : 0) * ld;
        double2 w = make_double2(0.0, 0.0);
        if (act)
          for (int i = k + gl; i < m; i += LPC) w = cconjfma(vbuf[i - k], col[i], w);
#pragma unroll
        for (int o = LPC / 2; o > 0; o >>= 1) {
          w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
          w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
        }
        w = make_double2(w.x * tau, w.y * tau);
        double ns = 0.0;
        if (act)
          for (int i = k + gl; i < m; i += LPC) {
            const double2 c = cfms(vbuf[i - k], w, col[i]);
            col[i] = c;
            if (i > k) ns = cabs2_acc(c, ns);
          }
#pragma unroll
        for (int o = LPC / 2; o > 0; o >>= 1) ns += __shfl_xor_sync(0xffffffffu, ns, o);
        if (act && gl == 0) norms[j] = sqrt(ns);
      }
    };
    if (a.max_m >= 128) apply_cols(std::integral_constant<int, 16>{});
    else apply_cols(std::integral_constant<int, 8>{});
    if (rank == owner && tid == 0) M[k + (long long)p * ld] = s_alpha;
    // the owner rewrites vbuf only after the next step's first cluster barrier,
    // which every reader of this step's v passes after finishing with it
    __syncthreads();
    ++k;
  }
  const int r = k;
  if (rank == 0 && tid == 0) {
    a.rank[jb.out_idx] = r;
    a.ref[jb.out_idx] = ref < 0.0 ? 0.0 : ref;
  }
  if (rank == 0)
    for (int i = tid; i < r; i += kThreads) perm_out[i] = order[i];
  // T = R11^{-1} R12, R11(a, b) = M(a, order[b]); one warp per owned remaining column
  double2* inv = vbuf;
  cl.sync();  // every block is done reading other blocks' shared memory
  for (int i = tid; i < r; i += kThreads) inv[i] = cinv(M[i + (long long)order[i] * ld]);
  __syncthreads();
  double2* T = a.tbuf + jb.t_off;
  for (int j = rank + C * warp; j < n; j += C * kWarps) {
    if (done[j]) continue;
    // position of j among the remaining columns (increasing index)
    int before = 0;
    for (int i = lane; i < j; i += 32) before += done[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
    const int c = j - before;
    if (lane == 0) perm_out[r + c] = j;
    if (r == 0) continue;
    double2* t = T + (long long)c * r;
    const double2* col = M + (long long)j * ld;
    for (int i = lane; i < r; i += 32) t[i] = col[i];
    __syncwarp();
    for (int i = r - 1; i >= 0; --i) {
      const double2 ti = cmul(t[i], inv[i]);
      __syncwarp();
      if (lane == 0) t[i] = ti;
      const double2* ri = M + (long long)order[i] * ld;
      for (int l = lane; l < i; l += 32) t[l] = cfms(ri[l], ti, t[l]);
      __syncwarp();
    }
  }
}

}  // namespace

// Cluster size for a launch: enough blocks per matrix to spread few large IDs
// over the SMs, at most 16, and at least 8 columns per block.
int cpqr_cluster_size(int njobs, int max_n) {
  int c = 1;
  while (c < 16 && njobs * c <= device_sm_count() && max_n >= 16 * c) c *= 2;
  return c;
}

cudaError_t launch_cpqr(const IdLaunch& a, cudaStream_t s) {
  if (a.njobs <= 0) return cudaSuccess;
  const size_t smem = (size_t)a.max_m * sizeof(double2) + (size_t)a.max_n * (sizeof(double) + 2 * sizeof(int));
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(cpqr_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int c = cpqr_cluster_size(a.njobs, a.max_n);
  while (c > 1 && c > a.cluster_max) c /= 2;
  if (c > 8) {
    if (cudaFuncSetAttribute(cpqr_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      c = 8;
    }
  }
  for (;;) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.njobs * c, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, cpqr_cluster_kernel, a);
    if (e == cudaSuccess) symhss::count_launches(1);
    if (e == cudaSuccess || c == 1) return e;
    cudaGetLastError();  // e.g. the cluster size is not supported: retry smaller
    c /= 2;
  }
}

}  // namespace symhss
