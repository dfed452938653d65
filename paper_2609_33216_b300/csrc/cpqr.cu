// Batched column interpolative decomposition by Householder QR with column
// pivoting (Sec. 4.1: the ID of each half of the proxy matrix M_R).
//
// One thread block per matrix (8 warps).  The matrix stays in global memory
// (it is L2-resident at these sizes); the Householder vector of the current step
// is staged in shared memory.  Step k:
//   1. pivot = column of largest remaining norm (ties to the lowest index);
//   2. stop if that norm <= tol * (first pivot norm) (tolerance mode) or after
//      `fixed` steps (fixed-rank mode);
//   3. swap it to position k, build the reflector H = I - tau v v^H with
//      H x = alpha e_1, |alpha| = |x|;
//   4. apply H to every trailing column (one warp per column) and, in the same
//      pass, recompute that column's remaining norm exactly.
// Afterwards T = R11^{-1} R12 is obtained by back substitution, one warp per
// column of R12.  The permutation and rank are written out; the matrix is left
// holding R in its upper triangle, so a later launch can continue the
// factorisation from step `start` (used to raise a rank to a prescribed value).
#include "common.cuh"

namespace symhss {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

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

__global__ void __launch_bounds__(kThreads) cpqr_kernel(const IdLaunch a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const IdJob jb = a.jobs[blockIdx.x];
  double2* vbuf = reinterpret_cast<double2*>(smem_raw);                 // max_m
  double* norms = reinterpret_cast<double*>(vbuf + a.max_m);            // max_n
  int* sperm = reinterpret_cast<int*>(norms + a.max_n);                 // max_n
  __shared__ double red[kWarps];
  __shared__ int redi[kWarps];
  __shared__ int s_piv;
  __shared__ double s_pv, s_tau;
  __shared__ double2 s_alpha;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = jb.m, n = jb.n, ld = jb.ld;
  if (m > a.max_m || n > a.max_n || m < 0 || n < 0) {
    if (tid == 0) { atomicOr(a.status, ST_BAD_INDEX); a.rank[jb.out_idx] = 0; }
    return;
  }
  double2* M = a.mats + jb.m_off;
  int* perm_out = a.perm + jb.perm_off;
  for (int j = tid; j < n; j += kThreads) sperm[j] = (jb.start == 0) ? j : perm_out[j];
  int kmax = min(m, n);
  if (jb.fixed >= 0) kmax = min(kmax, jb.fixed);
  int k = jb.start;
  // remaining norms of columns j >= k over rows k..m-1
  for (int j = k + warp; j < n; j += kWarps) {
    const double2* col = M + (long long)j * ld;
    double s = 0.0;
    for (int i = k + lane; i < m; i += 32) s += cabs2(col[i]);
    s = warp_sum(s);
    if (lane == 0) norms[j] = sqrt(s);
  }
  double ref = (jb.start == 0) ? -1.0 : a.ref[jb.out_idx];
  __syncthreads();

  while (k < kmax) {
    // 1. pivot
    double bv = -1.0;
    int bi = n;
    for (int j = k + tid; j < n; j += kThreads) {
      const double v = norms[j];
      if (v > bv || (v == bv && j < bi)) { bv = v; bi = j; }
    }
    warp_argmax(bv, bi);
    if (lane == 0) { red[warp] = bv; redi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      bv = lane < kWarps ? red[lane] : -1.0;
      bi = lane < kWarps ? redi[lane] : n;
      warp_argmax(bv, bi);
      if (lane == 0) { s_piv = bi; s_pv = bv; }
    }
    __syncthreads();
    const int p = s_piv;
    const double pv = s_pv;
    if (ref < 0.0) ref = pv;
    // 2. stop
    if (pv == 0.0) break;
    if (jb.fixed < 0 && pv <= a.tol * ref) break;
    // 3. swap columns k and p
    if (p != k) {
      double2* ck = M + (long long)k * ld;
      double2* cp = M + (long long)p * ld;
      for (int i = tid; i < m; i += kThreads) {
        const double2 t = ck[i];
        ck[i] = cp[i];
        cp[i] = t;
      }
      if (tid == 0) {
        const double tn = norms[k]; norms[k] = norms[p]; norms[p] = tn;
        const int tp = sperm[k]; sperm[k] = sperm[p]; sperm[p] = tp;
      }
    }
    __syncthreads();
    // Householder vector of column k, rows k..m-1
    const double2* ck = M + (long long)k * ld;
    double s = 0.0;
    for (int i = k + tid; i < m; i += kThreads) {
      const double2 x = ck[i];
      vbuf[i - k] = x;
      s += cabs2(x);
    }
    const double sigma2 = block_sum(s, red);
    if (tid == 0) {
      const double sigma = sqrt(sigma2);
      const double2 x0 = vbuf[0];
      const double ax0 = sqrt(cabs2(x0));
      const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
      s_alpha = make_double2(-ph.x * sigma, -ph.y * sigma);
      vbuf[0] = make_double2(ph.x * (ax0 + sigma), ph.y * (ax0 + sigma));
      const double vn2 = 2.0 * sigma * (sigma + ax0);
      s_tau = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
    }
    __syncthreads();
    const double tau = s_tau;
    // 4. apply to trailing columns, recompute their remaining norms
    for (int j = k + 1 + warp; j < n; j += kWarps) {
      double2* col = M + (long long)j * ld;
      double2 w = make_double2(0.0, 0.0);
      for (int i = k + lane; i < m; i += 32) w = cadd(w, cconjmul(vbuf[i - k], col[i]));
      w = warp_csum(w);
      w = make_double2(w.x * tau, w.y * tau);
      double ns = 0.0;
      for (int i = k + lane; i < m; i += 32) {
        const double2 c = cfms(vbuf[i - k], w, col[i]);
        col[i] = c;
        if (i > k) ns += cabs2(c);
      }
      ns = warp_sum(ns);
      if (lane == 0) norms[j] = sqrt(ns);
    }
    if (tid == 0) M[k + (long long)k * ld] = s_alpha;
    __syncthreads();
    ++k;
  }
  const int r = k;
  if (tid == 0) {
    a.rank[jb.out_idx] = r;
    a.ref[jb.out_idx] = ref < 0.0 ? 0.0 : ref;
  }
  for (int j = tid; j < n; j += kThreads) perm_out[j] = sperm[j];
  // T = R11^{-1} R12 (r x (n - r), leading dimension r); barriers stay unconditional
  double2* inv = vbuf;  // r <= min(m, n) <= max_m
  for (int i = tid; i < r; i += kThreads) inv[i] = cinv(M[i + (long long)i * ld]);
  __syncthreads();
  double2* T = a.tbuf + jb.t_off;
  for (int j = r + warp; r > 0 && j < n; j += kWarps) {
    double2* t = T + (long long)(j - r) * r;
    const double2* col = M + (long long)j * ld;
    for (int i = lane; i < r; i += 32) t[i] = col[i];
    __syncwarp();
    for (int i = r - 1; i >= 0; --i) {
      const double2 ti = cmul(t[i], inv[i]);
      __syncwarp();
      if (lane == 0) t[i] = ti;
      const double2* ri = M + (long long)i * ld;
      for (int l = lane; l < i; l += 32) t[l] = cfms(ri[l], ti, t[l]);
      __syncwarp();
    }
  }
}

}  // namespace

cudaError_t launch_cpqr(const IdLaunch& a, cudaStream_t s) {
  if (a.njobs <= 0) return cudaSuccess;
  const size_t smem = (size_t)a.max_m * sizeof(double2) + (size_t)a.max_n * (sizeof(double) + sizeof(int));
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(cpqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cpqr_kernel<<<a.njobs, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace symhss
