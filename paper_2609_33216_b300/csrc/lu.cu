// Triangular solves with the factors of the batched LU (lu_blocked.cu): the
// solves of Sec. 4.2 (X = D^{-1} L, Atilde = (R X)^{-1}, g = D^{-1} f, root).
// One warp per right-hand side; the permuted column is held in shared memory
// while the unit-lower and upper triangular solves run.
#include "common.cuh"

namespace symhss {

namespace {

constexpr int kRsWarps = 4;

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
