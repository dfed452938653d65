// Interpolation residual of column IDs.  A sketched ID selects its skeleton J and T from
// rows of Y = Omega M (Sec. 4.1 with a randomized range finder); the runtime points this
// check at sketch rows the ID did not see, where the residual of column c is
// Omega_h (m_c - M_J t_c): its norm estimates the residual on M itself (the a-posteriori
// estimator of Halko, Martinsson and Tropp).  The ID is accepted only if the largest
// residual is at most the ID tolerance times the largest column norm of the same rows --
// the bound the plain ID meets by construction -- and is otherwise redone as a plain ID
// of M.  The kernel itself computes the ratio for whatever rows it is given.
//
// kCheckSplit blocks per ID, each taking every kCheckSplit-th group of columns: warps own
// columns; a lane walks the rows of its warp's column, so reads of M are coalesced;
// per-column sums of squares are reduced with shuffles.  The blocks' largest sums meet in
// two 64-bit maxima per ID (the bit patterns of non-negative doubles order like the values),
// and a second launch forms the ratio.  (One block per ID left the top levels' few IDs, whose
// columns each take an r-step dependent chain, on a few SMs.)
#include "common.cuh"

namespace symhss {

namespace {

constexpr int kCheckThreads = 256;
constexpr int kCheckSplit = 8;

__global__ void __launch_bounds__(kCheckThreads) id_check_kernel(const double2* mats, const double2* tbuf,
                                                                 const int* perm, const int* rank,
                                                                 const CheckJob* jobs,
                                                                 unsigned long long* acc) {
  __shared__ double s_max[2][kCheckThreads / 32];
  const CheckJob jb = jobs[blockIdx.x];
  const double2* M = mats + jb.m_off;
  const double2* T = tbuf + jb.t_off;
  const int* pm = perm + jb.perm_off;
  const int r = min(max(rank[jb.rank_idx], 0), jb.n);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kCheckThreads / 32;
  const int c0 = warp + nw * blockIdx.y, cs = nw * kCheckSplit;
  double ref = 0.0, res = 0.0;
  // largest column norm of M
  for (int c = c0; c < jb.n; c += cs) {
    const double2* col = M + (long long)c * jb.ld;
    double ss = 0.0;
    for (int i = lane; i < jb.m; i += 32) ss = fma(col[i].x, col[i].x, fma(col[i].y, col[i].y, ss));
    ss = warp_sum(ss);
    ref = fmax(ref, ss);
  }
  // residual of every non-skeleton column
  for (int c = r + c0; c < jb.n; c += cs) {
    const double2* col = M + (long long)pm[c] * jb.ld;
    const double2* tc = T + (long long)(c - r) * r;
    double ss = 0.0;
    for (int i = lane; i < jb.m; i += 32) {
      double2 e = col[i];
      for (int k = 0; k < r; ++k) e = cfms(M[i + (long long)pm[k] * jb.ld], tc[k], e);
      ss = fma(e.x, e.x, fma(e.y, e.y, ss));
    }
    ss = warp_sum(ss);
    res = fmax(res, ss);
  }
  if (lane == 0) { s_max[0][warp] = ref; s_max[1][warp] = res; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < nw; ++w) { a = fmax(a, s_max[0][w]); b = fmax(b, s_max[1][w]); }
    atomicMax(&acc[2 * jb.out], (unsigned long long)__double_as_longlong(a));
    atomicMax(&acc[2 * jb.out + 1], (unsigned long long)__double_as_longlong(b));
  }
}

__global__ void id_check_ratio_kernel(const unsigned long long* acc, int n, double* ratio) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = __longlong_as_double((long long)acc[2 * i]), b = __longlong_as_double((long long)acc[2 * i + 1]);
  ratio[i] = a > 0.0 ? sqrt(b / a) : 0.0;
}

}  // namespace

cudaError_t launch_id_check(const double2* mats, const double2* tbuf, const int* perm, const int* rank,
                            const CheckJob* jobs, int njobs, double* ratio, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  // the maxima after the njobs ratios (the caller's buffer holds 3 njobs doubles)
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(ratio + njobs);
  cudaError_t e = cudaMemsetAsync(acc, 0, 2 * (size_t)njobs * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  id_check_kernel<<<dim3(njobs, kCheckSplit), kCheckThreads, 0, s>>>(mats, tbuf, perm, rank, jobs, acc);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  id_check_ratio_kernel<<<(njobs + 127) / 128, 128, 0, s>>>(acc, njobs, ratio);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symhss

// ---- exact residual on the proxy matrix, with the product on the tensor cores ----------
// For each checked ID of M (m x n): G1 = M[:, perm[0:r]] and G2 = M[:, perm[r:n]] are
// gathered, G2 -= G1 T runs on the tensor cores (zgemm_tc.cu), and the ratio of G2's largest
// column norm to M's is taken.

namespace symhss {

namespace {

__global__ void __launch_bounds__(256) gather_cols_kernel(const double2* mats, const int* perm,
                                                           const GatherJob* jobs, const int2* work, double2* g) {
  const int2 w = work[blockIdx.x];
  const GatherJob jb = jobs[w.x];
  const int c = w.y;
  const int src = perm[jb.perm_off + c];
  if (src < 0 || src >= jb.n) return;  // a permutation entry out of range: leave the column unset
  const double2* col = mats + jb.m_off + (long long)src * jb.ld;
  double2* dst = g + (c < jb.r ? jb.g1_off + (long long)c * jb.m : jb.g2_off + (long long)(c - jb.r) * jb.m);
  for (int i = threadIdx.x; i < jb.m; i += blockDim.x) dst[i] = col[i];
}

__global__ void __launch_bounds__(256) ratio_kernel(const double2* mats, const double2* g, const GatherJob* jobs,
                                                    const int* outs, double* ratio) {
  __shared__ double s_max[2][8];
  const GatherJob jb = jobs[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double ref = 0.0, res = 0.0;
  for (int c = warp; c < jb.n; c += 8) {
    const double2* col = mats + jb.m_off + (long long)c * jb.ld;
    double ss = 0.0;
    for (int i = lane; i < jb.m; i += 32) ss = fma(col[i].x, col[i].x, fma(col[i].y, col[i].y, ss));
    ref = fmax(ref, warp_sum(ss));
  }
  for (int c = warp; c < jb.n - jb.r; c += 8) {
    const double2* col = g + jb.g2_off + (long long)c * jb.m;
    double ss = 0.0;
    for (int i = lane; i < jb.m; i += 32) ss = fma(col[i].x, col[i].x, fma(col[i].y, col[i].y, ss));
    res = fmax(res, warp_sum(ss));
  }
  if (lane == 0) { s_max[0][warp] = ref; s_max[1][warp] = res; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < 8; ++q) { a = fmax(a, s_max[0][q]); b = fmax(b, s_max[1][q]); }
    ratio[outs[blockIdx.x]] = a > 0.0 ? sqrt(b / a) : 0.0;
  }
}

}  // namespace

cudaError_t launch_gather_cols(const double2* mats, const int* perm, const GatherJob* jobs, const int2* work,
                               int nwork, double2* g, cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  gather_cols_kernel<<<nwork, 256, 0, s>>>(mats, perm, jobs, work, g);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_residual_ratio(const double2* mats, const double2* g, const GatherJob* jobs, const int* outs,
                                  int njobs, double* ratio, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  ratio_kernel<<<njobs, 256, 0, s>>>(mats, g, jobs, outs, ratio);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symhss
