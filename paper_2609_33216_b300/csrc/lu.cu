// Batched dense LU with partial pivoting and the matching triangular solves
// (the diagonal-block factorisations of Sec. 4.2: D_tau = P L U, X = D^{-1} L,
// Atilde = (R X)^{-1}, root block).
//
// getrf: one thread block per matrix, right-looking and unblocked; the pivot
// column and row of each step are staged in shared memory and the trailing
// update runs one warp per column with lanes over rows (coalesced).
// getrs: one warp per right-hand side; the permuted column is held in shared
// memory while the unit-lower and upper triangular solves run.
#include "common.cuh"

namespace symhss {

namespace {

constexpr int kLuThreads = 256;
constexpr int kLuWarps = kLuThreads / 32;
constexpr int kRsWarps = 4;

__global__ void __launch_bounds__(kLuThreads) getrf_kernel(const LuLaunch a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* urow = reinterpret_cast<double2*>(smem_raw);
  double2* lcol = urow + a.max_n;
  __shared__ double red[kLuWarps];
  __shared__ int redi[kLuWarps];
  __shared__ int s_piv;
  __shared__ double s_pv;
  const LuJob jb = a.jobs[blockIdx.x];
  const int n = jb.n, ld = jb.ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (n > a.max_n || n < 0) {
    if (tid == 0) { atomicOr(a.status, ST_BAD_INDEX); a.info[jb.info_idx] = -1; }
    return;
  }
  double2* A = a.base + jb.a_off;
  int* piv = a.piv + jb.piv_off;
  int info = 0;
  for (int k = 0; k < n; ++k) {
    double bv = -1.0;
    int bi = n;
    const double2* ck = A + (long long)k * ld;
    for (int i = k + tid; i < n; i += kLuThreads) {
      const double v = cabs1(ck[i]);
      if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
    }
    warp_argmax(bv, bi);
    if (lane == 0) { red[warp] = bv; redi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      bv = lane < kLuWarps ? red[lane] : -1.0;
      bi = lane < kLuWarps ? redi[lane] : n;
      warp_argmax(bv, bi);
      if (lane == 0) { s_piv = bi; s_pv = bv; }
    }
    __syncthreads();
    const int p = s_piv;
    if (tid == 0) piv[k] = p;
    if (s_pv == 0.0) {  // exactly singular column: record, leave the column, continue
      if (info == 0) info = k + 1;
      __syncthreads();
      continue;
    }
    if (p != k) {
      for (int j = tid; j < n; j += kLuThreads) {
        double2* c = A + (long long)j * ld;
        const double2 t = c[k];
        c[k] = c[p];
        c[p] = t;
      }
    }
    __syncthreads();
    const double2 inv = cinv(A[k + (long long)k * ld]);
    for (int i = k + 1 + tid; i < n; i += kLuThreads) {
      const double2 l = cmul(A[i + (long long)k * ld], inv);
      A[i + (long long)k * ld] = l;
      lcol[i] = l;
    }
    for (int j = k + 1 + tid; j < n; j += kLuThreads) urow[j] = A[k + (long long)j * ld];
    __syncthreads();
    for (int j = k + 1 + warp; j < n; j += kLuWarps) {
      const double2 u = urow[j];
      double2* c = A + (long long)j * ld;
      for (int i = k + 1 + lane; i < n; i += 32) c[i] = cfms(lcol[i], u, c[i]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    a.info[jb.info_idx] = info;
    if (info != 0) atomicOr(a.status, ST_SINGULAR);
  }
}

__global__ void __launch_bounds__(kRsWarps * 32) getrs_kernel(const RsLaunch a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RsJob jb = a.jobs[blockIdx.x];
  const int n = jb.n;
  if (n > a.max_n || n < 0) return;
  int* perm = reinterpret_cast<int*>(smem_raw);
  double2* cols = reinterpret_cast<double2*>(smem_raw + ((n * sizeof(int) + 15) / 16) * 16);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int* piv = a.piv + jb.piv_off;
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k && p >= 0 && p < n) { const int t = perm[k]; perm[k] = perm[p]; perm[p] = t; }
    }
  }
  __syncthreads();
  const int c = blockIdx.y * kRsWarps + warp;
  if (c >= jb.nrhs) return;
  const double2* A = a.abase + jb.a_off;
  const int lda = jb.lda;
  double2* b = a.bbase + jb.b_off + (long long)c * jb.ldb;
  double2* sb = cols + (long long)warp * n;
  for (int i = lane; i < n; i += 32) sb[i] = b[perm[i]];
  __syncwarp();
  for (int k = 0; k < n; ++k) {  // unit lower
    const double2 bk = sb[k];
    const double2* lk = A + (long long)k * lda;
    for (int i = k + 1 + lane; i < n; i += 32) sb[i] = cfms(lk[i], bk, sb[i]);
    __syncwarp();
  }
  for (int k = n - 1; k >= 0; --k) {  // upper
    const double2* uk = A + (long long)k * lda;
    const double2 bk = cmul(sb[k], cinv(uk[k]));
    __syncwarp();
    if (lane == 0) sb[k] = bk;
    for (int i = lane; i < k; i += 32) sb[i] = cfms(uk[i], bk, sb[i]);
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) b[i] = sb[i];
}

}  // namespace

cudaError_t launch_getrf(const LuLaunch& a, cudaStream_t s) {
  if (a.njobs <= 0) return cudaSuccess;
  const size_t smem = 2 * (size_t)a.max_n * sizeof(double2);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(getrf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  getrf_kernel<<<a.njobs, kLuThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_getrs(const RsLaunch& a, cudaStream_t s) {
  const int max_n = a.max_n;
  if (a.njobs <= 0 || a.max_rhs <= 0) return cudaSuccess;
  const size_t smem = ((max_n * sizeof(int) + 15) / 16) * 16 + (size_t)kRsWarps * max_n * sizeof(double2);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(getrs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.njobs, (a.max_rhs + kRsWarps - 1) / kRsWarps);
  getrs_kernel<<<grid, kRsWarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace symhss
