// Triangular solves with the factors of the batched LU (lu_blocked.cu): the
// solves of Sec. 4.2 (X = D^{-1} L, Atilde = (R X)^{-1}, g = D^{-1} f, root).
//
// Many right-hand sides (factorisation): one warp per right-hand side, up to 8 per
// block; the permuted column and the inverted diagonal of U live in shared memory.
// Few right-hand sides (solve phase): one block per right-hand side; the column is
// processed in 32-row blocks -- one warp solves the 32 x 32 triangle with register
// shuffles, then every thread of the block updates the rows below (above, for U).
// FP64 with many right-hand sides and n > 64 (the factorisation's X = D^{-1} L and Atilde):
// blocked by 64 rows -- an FP64 solve with each diagonal block (one warp per right-hand
// side) and the update of the other rows, X[rows] -= (block column of L or U) X[block], on
// the tensor cores (zgemm_tc.cu).
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace symhss {

namespace {

constexpr int kRsMaxWarps = 8;
constexpr int kCtaThreads = 256;

template <typename CT> __device__ __forceinline__ const CT* rs_a(const RsLaunch& a);
template <> __device__ __forceinline__ const double2* rs_a<double2>(const RsLaunch& a) { return a.abase; }
template <> __device__ __forceinline__ const float2* rs_a<float2>(const RsLaunch& a) { return a.abase32; }
template <typename CT> __device__ __forceinline__ CT* rs_b(const RsLaunch& a);
template <> __device__ __forceinline__ double2* rs_b<double2>(const RsLaunch& a) { return a.bbase; }
template <> __device__ __forceinline__ float2* rs_b<float2>(const RsLaunch& a) { return a.bbase32; }

// perm = composition of the recorded row interchanges (thread 0, sequential)
__device__ __forceinline__ void build_perm(int* perm, const int* piv, int n) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k && p >= 0 && p < n) { const int t = perm[k]; perm[k] = perm[p]; perm[p] = t; }
    }
  }
}

// the solve's row permutation into shared memory: copied from the one the LU kept, else
// composed from piv by thread 0; the caller synchronises the block before using it
__device__ __forceinline__ void load_perm(int* perm, const RsLaunch& a, const RsJob& jb, int n) {
  if (a.perm) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = a.perm[jb.piv_off + i];
  } else {
    build_perm(perm, a.piv + jb.piv_off, n);
  }
}

// ---- 32-row diagonal blocks solved through the inverses of their 8 x 8 diagonal sub-blocks
// (the serial chain of a 32-step substitution becomes four short matrix-vector steps)

// Column j of the inverse of sub-block s (rows and columns 8 s .. 8 s + 7) of a 32 x 32 diagonal
// block (column-major `tri`, w valid rows): unit lower part (LOWER) or upper part with the
// diagonal reciprocals dinv (indexed by block row); written to inv[s * 64 + j * 8 + i].
template <bool LOWER>
__device__ __forceinline__ void inv8_column(const double2* tri, const double2* dinv, double2* inv, int w, int s,
                                            int j) {
  const int o = 8 * s;
  double2 y[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) y[i] = make_double2(0.0, 0.0);
  if (o + j < w) {
    if (LOWER) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (i == j) y[i] = make_double2(1.0, 0.0);
        if (i > j && o + i < w) {
          double2 acc = make_double2(0.0, 0.0);
#pragma unroll
          for (int k = 0; k < i; ++k)
            if (k >= j) acc = cfms(tri[(o + k) * 32 + o + i], y[k], acc);
          y[i] = acc;
        }
      }
    } else {
#pragma unroll
      for (int i = 7; i >= 0; --i) {
        if (i == j) y[i] = dinv[o + i];
        if (i < j) {
          double2 acc = make_double2(0.0, 0.0);
#pragma unroll
          for (int k = 1; k < 8; ++k)
            if (k > i && k <= j) acc = cfms(tri[(o + k) * 32 + o + i], y[k], acc);
          y[i] = cmul(acc, dinv[o + i]);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) inv[s * 64 + j * 8 + i] = y[i];
}

// sum of v over the 8 lanes of each aligned group of 8 (every lane of the warp takes part)
__device__ __forceinline__ double2 sum8(double2 v) {
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// xb[0 .. w) <- T^{-1} xb for the 32 x 32 diagonal block T (unit lower: LOWER; else upper), by
// all threads of the block (at least 256): per 8-row sub-block (top-down for L, bottom-up for
// U), y = inv_s x_s, then the rows of the sub-blocks still to come are updated with y.
template <bool LOWER>
__device__ __forceinline__ void block_solve32(double2* xb, const double2* tri, const double2* inv, int w) {
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int ss = 0; ss < 4; ++ss) {
    const int s = LOWER ? ss : 3 - ss;
    const int o = 8 * s;
    if (o >= w) continue;  // uniform
    double2 p = make_double2(0.0, 0.0);
    if (tid < 64) {
      const int i = tid >> 3, k = tid & 7;
      if ((LOWER ? k <= i : k >= i) && o + k < w && o + i < w) p = cmul(inv[s * 64 + k * 8 + i], xb[o + k]);
    }
    const double2 y = sum8(p);
    __syncthreads();  // every read of the sub-block's x before its new values
    if (tid < 64 && (tid & 7) == 0 && o + (tid >> 3) < w) xb[o + (tid >> 3)] = y;
    __syncthreads();
    const int rlo = LOWER ? o + 8 : 0, rhi = LOWER ? w : o;
    if (rhi > rlo) {  // uniform
      const int r = rlo + (tid >> 3), k = tid & 7;
      double2 q = make_double2(0.0, 0.0);
      if (r < rhi && o + k < w) q = cmul(tri[(o + k) * 32 + r], xb[o + k]);
      const double2 u = sum8(q);
      if (r < rhi && k == 0) xb[r] = make_double2(xb[r].x - u.x, xb[r].y - u.y);
    }
    __syncthreads();
  }
}

template <typename CT>
__global__ void getrs_kernel(const RsLaunch a, int warps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RsJob jb = a.jobs[blockIdx.x];
  const int n = jb.n;
  if (n > a.max_n || n < 0) return;  // uniform per block
  CT* dinv = reinterpret_cast<CT*>(smem_raw);
  CT* cols = dinv + a.max_n;
  int* perm = reinterpret_cast<int*>(cols + (size_t)warps * a.max_n);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const CT* A = rs_a<CT>(a) + jb.a_off;
  const int lda = jb.lda;
  load_perm(perm, a, jb, n);
  for (int i = threadIdx.x; i < n; i += blockDim.x) dinv[i] = cinv(A[i + (long long)i * lda]);
  __syncthreads();
  const int c = blockIdx.y * warps + warp;
  if (c >= jb.nrhs) return;
  CT* b = rs_b<CT>(a) + jb.b_off + (long long)c * jb.ldb;
  CT* sb = cols + (long long)warp * a.max_n;
  for (int i = lane; i < n; i += 32) sb[i] = b[perm[i]];
  __syncwarp();
  for (int k = 0; k < n; ++k) {  // unit lower
    const CT bk = sb[k];
    const CT* lk = A + (long long)k * lda;
    for (int i = k + 1 + lane; i < n; i += 32) sb[i] = cfms(lk[i], bk, sb[i]);
    __syncwarp();
  }
  for (int k = n - 1; k >= 0; --k) {  // upper
    const CT* uk = A + (long long)k * lda;
    const CT bk = cmul(sb[k], dinv[k]);
    __syncwarp();
    if (lane == 0) sb[k] = bk;
    for (int i = lane; i < k; i += 32) sb[i] = cfms(uk[i], bk, sb[i]);
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) b[i] = sb[i];
}

// rows [r0, r1) of x (stride kCtaThreads from r0 + tid) -= A[rows, kb .. kb + w) x[kb .. kb + w):
// for full 32-column blocks the loop is unrolled so that the 32 loads of a row are in
// flight together, and four partial sums shorten the FP64 dependency chain
template <typename CT>
__device__ __forceinline__ void cta_update_rows(const CT* A, int lda, CT* x, int kb, int w, int r0, int r1) {
  for (int i = r0 + (int)threadIdx.x; i < r1; i += kCtaThreads) {
    const CT* ai = A + i + (long long)kb * lda;
    CT acc0 = x[i], acc1 = make_c<CT>(0.0, 0.0), acc2 = acc1, acc3 = acc1;
    if (w == 32) {
#pragma unroll
      for (int q = 0; q < 32; q += 4) {
        acc0 = cfms(ai[(long long)q * lda], x[kb + q], acc0);
        acc1 = cfms(ai[(long long)(q + 1) * lda], x[kb + q + 1], acc1);
        acc2 = cfms(ai[(long long)(q + 2) * lda], x[kb + q + 2], acc2);
        acc3 = cfms(ai[(long long)(q + 3) * lda], x[kb + q + 3], acc3);
      }
    } else {
      for (int q = 0; q < w; ++q) acc0 = cfms(ai[(long long)q * lda], x[kb + q], acc0);
    }
    x[i] = cadd(cadd(acc0, acc1), cadd(acc2, acc3));
  }
}

template <typename CT>
__global__ void __launch_bounds__(kCtaThreads) getrs_cta_kernel(const RsLaunch a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ CT tri[32 * 32];  // the current 32 x 32 diagonal block, column-major
  const RsJob jb = a.jobs[blockIdx.x];
  const int n = jb.n;
  const int c = blockIdx.y;
  if (n > a.max_n || n < 0 || c >= jb.nrhs) return;  // uniform per block
  CT* x = reinterpret_cast<CT*>(smem_raw);
  CT* dinv = x + a.max_n;
  int* perm = reinterpret_cast<int*>(dinv + a.max_n);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const CT* A = rs_a<CT>(a) + jb.a_off;
  const int lda = jb.lda;
  CT* b = rs_b<CT>(a) + jb.b_off + (long long)c * jb.ldb;
  load_perm(perm, a, jb, n);
  // the reciprocals of U's diagonal, all at once: the serial 32-row solves below then
  // carry only multiplications on their dependency chain
  for (int i = tid; i < n; i += kCtaThreads) dinv[i] = cinv(A[i + (long long)i * lda]);
  __syncthreads();
  for (int i = tid; i < n; i += kCtaThreads) x[i] = b[perm[i]];
  // forward substitution with the unit lower factor, 32 rows at a time; the diagonal
  // block is staged in shared memory so that warp 0's serial solve waits on no L2 load
  for (int kb = 0; kb < n; kb += 32) {
    const int w = min(32, n - kb);
    for (int e = tid; e < 32 * w; e += kCtaThreads) {
      const int r = e & 31, q = e >> 5;
      tri[e] = r < w ? A[kb + r + (long long)(kb + q) * lda] : make_c<CT>(0.0, 0.0);
    }
    __syncthreads();
    if (warp == 0) {
      CT xr = lane < w ? x[kb + lane] : make_c<CT>(0.0, 0.0);
      for (int q = 0; q < w; ++q) {
        const CT xq = make_c<CT>(__shfl_sync(0xffffffffu, xr.x, q), __shfl_sync(0xffffffffu, xr.y, q));
        if (lane > q && lane < w) xr = cfms(tri[q * 32 + lane], xq, xr);
      }
      if (lane < w) x[kb + lane] = xr;
    }
    __syncthreads();
    cta_update_rows(A, lda, x, kb, w, kb + w, n);
    __syncthreads();
  }
  // back substitution with the upper factor, 32 rows at a time from the bottom
  for (int kb = ((n - 1) / 32) * 32; n > 0 && kb >= 0; kb -= 32) {
    const int w = min(32, n - kb);
    for (int e = tid; e < 32 * w; e += kCtaThreads) {
      const int r = e & 31, q = e >> 5;
      tri[e] = r < w ? A[kb + r + (long long)(kb + q) * lda] : make_c<CT>(0.0, 0.0);
    }
    __syncthreads();
    if (warp == 0) {
      CT xr = lane < w ? x[kb + lane] : make_c<CT>(0.0, 0.0);
      const CT dl = lane < w ? dinv[kb + lane] : make_c<CT>(0.0, 0.0);
      for (int q = w - 1; q >= 0; --q) {
        if (lane == q) xr = cmul(xr, dl);
        const CT xq = make_c<CT>(__shfl_sync(0xffffffffu, xr.x, q), __shfl_sync(0xffffffffu, xr.y, q));
        if (lane < q) xr = cfms(tri[q * 32 + lane], xq, xr);
      }
      if (lane < w) x[kb + lane] = xr;
    }
    __syncthreads();
    cta_update_rows(A, lda, x, kb, w, 0, kb);
    __syncthreads();
  }
  for (int i = tid; i < n; i += kCtaThreads) b[i] = x[i];
}

// Few right-hand sides and few large blocks (the top tree levels of the solve phase): one
// thread-block cluster of C blocks per (matrix, right-hand side), so that the FP64 updates of a
// block's rows spread over C SMs.  The 32-row blocks of the matrix belong to the cluster's
// members in turn (block b to member b % C), which preload their diagonal 32 x 32 blocks
// (unit L below the diagonal, U on and above it) and the inverses of their 8 x 8 diagonal
// sub-blocks.  Forward: the owner of block b solves its triangle with all its threads
// (block_solve32), one cluster barrier publishes the 32 values, and
// every member reads them through distributed shared memory and updates its own rows below;
// backward likewise with U, from the last block.  The arithmetic of every row is that of the
// one-block kernel up to the order of the partial sums.
constexpr int kClThreads = 256;

__global__ void __launch_bounds__(kClThreads) getrs_cluster_kernel(const RsLaunch a, int nbown) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double2 xk[32];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int grp = blockIdx.x / C;
  const int jidx = grp / a.max_rhs, c = grp - jidx * a.max_rhs;
  const RsJob jb = a.jobs[jidx];
  const int n = jb.n;
  const int nb = (n + 31) / 32;
  // uniform over the cluster (every member has the same job and right-hand side)
  if (n > a.max_n || n <= 0 || c >= jb.nrhs || (nb + C - 1) / C > nbown) return;
  double2* x = reinterpret_cast<double2*>(smem_raw);          // max_n: the own rows are current
  double2* tri = x + a.max_n;                                  // nbown x 32 x 32, column-major
  double2* dinv = tri + (size_t)nbown * 1024;                  // nbown x 32
  double2* inv = dinv + (size_t)nbown * 32;                    // nbown x (L, U) x 4 x 8 x 8
  int* perm = reinterpret_cast<int*>(inv + (size_t)nbown * 512);  // max_n
  const int tid = threadIdx.x;
  const double2* A = a.abase + jb.a_off;
  const int lda = jb.lda;
  double2* b = a.bbase + jb.b_off + (long long)c * jb.ldb;
  load_perm(perm, a, jb, n);
  // own diagonal blocks and the reciprocals of their U diagonal
  for (int t = 0; rank + t * C < nb; ++t) {
    const int kb = (rank + t * C) * 32, w = min(32, n - kb);
    for (int e = tid; e < 1024; e += kClThreads) {
      const int r = e & 31, q = e >> 5;
      tri[t * 1024 + e] = (r < w && q < w) ? A[kb + r + (long long)(kb + q) * lda] : make_double2(0.0, 0.0);
    }
    if (tid < w) dinv[t * 32 + tid] = cinv(A[kb + tid + (long long)(kb + tid) * lda]);
  }
  __syncthreads();
  // the inverses of the 8 x 8 diagonal sub-blocks of the own blocks (one thread per column)
  const int nown = (nb - rank + C - 1) / C;
  for (int task = tid; task < nown * 64; task += kClThreads) {
    const int t = task >> 6, r = task & 63;
    const int w = min(32, n - (rank + t * C) * 32);
    if (r < 32) inv8_column<true>(tri + t * 1024, nullptr, inv + t * 512, w, r >> 3, r & 7);
    else inv8_column<false>(tri + t * 1024, dinv + t * 32, inv + t * 512 + 256, w, (r - 32) >> 3, r & 7);
  }
  __syncthreads();
  // x = P b on the own rows
  for (int bb = rank; bb < nb; bb += C)
    for (int i = bb * 32 + tid; i < min(n, bb * 32 + 32); i += kClThreads) x[i] = b[perm[i]];
  __syncthreads();
  // Update of the own rows of blocks [blo, bhi): x_i -= A[i, kb .. kb + w) xk, four threads per
  // row (eight columns each, two chains), 64 rows per pass.  The operands of the first pass do
  // not depend on the block's solution: they are loaded before the cluster barrier, while the
  // owner solves its triangle.
  struct Pass { int i; bool live; };
  auto pass_row = [&](int blo, int bhi, int base) -> Pass {
    const int first = blo + ((rank - blo) % C + C) % C;  // first own block >= blo
    const int ri = base + (tid >> 2);
    const int bidx = first + (ri >> 5) * C;
    const int i = bidx * 32 + (ri & 31);
    return Pass{i, bidx < bhi && i < n};
  };
  auto pass_any = [&](int blo, int bhi, int base) {  // uniform: does this pass hold own rows?
    const int first = blo + ((rank - blo) % C + C) % C;
    return first + (base >> 5) * C < bhi;
  };
  auto load_ops = [&](const Pass& p, int kb, int w, double2 av[8]) {
    const int part = tid & 3;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int q = part * 8 + e;
      av[e] = (p.live && q < w) ? A[p.i + (long long)(kb + q) * lda] : make_double2(0.0, 0.0);
    }
  };
  auto apply = [&](const Pass& p, const double2 av[8]) {
    const int part = tid & 3;
    double2 acc0 = make_double2(0.0, 0.0), acc1 = acc0;
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      acc0 = cfms(av[e], xk[part * 8 + e], acc0);
      acc1 = cfms(av[e + 1], xk[part * 8 + e + 1], acc1);
    }
    double2 acc = cadd(acc0, acc1);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
    if (p.live && part == 0) x[p.i] = make_double2(x[p.i].x + acc.x, x[p.i].y + acc.y);
  };
  auto update_rest = [&](int blo, int bhi, int kb, int w) {  // passes after the first
    for (int base = kClThreads / 4; pass_any(blo, bhi, base); base += kClThreads / 4) {
      const Pass p = pass_row(blo, bhi, base);
      double2 av[8];
      load_ops(p, kb, w, av);
      apply(p, av);
    }
  };
  // forward substitution with the unit lower factor
  for (int bk = 0; bk < nb; ++bk) {
    const int kb = bk * 32, w = min(32, n - kb), owner = bk % C;
    const bool upd = bk + 1 < nb && pass_any(bk + 1, nb, 0);
    Pass p0{0, false};
    double2 av[8];
    if (upd) {
      p0 = pass_row(bk + 1, nb, 0);
      load_ops(p0, kb, w, av);
    }
    if (rank == owner) block_solve32<true>(x + kb, tri + (bk / C) * 1024, inv + (bk / C) * 512, w);
    cl.sync();
    if (tid < 32) xk[tid] = tid < w ? cl.map_shared_rank(x, owner)[kb + tid] : make_double2(0.0, 0.0);
    __syncthreads();
    if (upd) {
      apply(p0, av);
      update_rest(bk + 1, nb, kb, w);
    }
    __syncthreads();
  }
  // back substitution with the upper factor, from the last block
  for (int bk = nb - 1; bk >= 0; --bk) {
    const int kb = bk * 32, w = min(32, n - kb), owner = bk % C;
    const bool upd = bk > 0 && pass_any(0, bk, 0);
    Pass p0{0, false};
    double2 av[8];
    if (upd) {
      p0 = pass_row(0, bk, 0);
      load_ops(p0, kb, w, av);
    }
    if (rank == owner) block_solve32<false>(x + kb, tri + (bk / C) * 1024, inv + (bk / C) * 512 + 256, w);
    cl.sync();
    if (tid < 32) xk[tid] = tid < w ? cl.map_shared_rank(x, owner)[kb + tid] : make_double2(0.0, 0.0);
    __syncthreads();
    if (upd) {
      apply(p0, av);
      update_rest(0, bk, kb, w);
    }
    __syncthreads();
  }
  for (int bb = rank; bb < nb; bb += C)
    for (int i = bb * 32 + tid; i < min(n, bb * 32 + 32); i += kClThreads) b[i] = x[i];
  cl.sync();  // no member reads another's shared memory after this point
}

// ---- blocked solve with tensor-core updates (FP64, many right-hand sides) ----------------
constexpr int kBlk = 64;  // largest diagonal block of the blocked solve (shared-memory stride)

// b <- P b for every right-hand side (one warp per column, the column staged in shared memory)
__global__ void permute_kernel(const RsLaunch a, int warps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RsJob jb = a.jobs[blockIdx.x];
  const int n = jb.n;
  if (n > a.max_n || n < 0) return;  // uniform per block
  double2* cols = reinterpret_cast<double2*>(smem_raw);
  int* perm = reinterpret_cast<int*>(cols + (size_t)warps * a.max_n);
  load_perm(perm, a, jb, n);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * warps + warp;
  if (c >= jb.nrhs) return;
  double2* b = a.bbase + jb.b_off + (long long)c * jb.ldb;
  double2* sb = cols + (long long)warp * a.max_n;
  for (int i = lane; i < n; i += 32) sb[i] = b[perm[i]];
  __syncwarp();
  for (int i = lane; i < n; i += 32) b[i] = sb[i];
}

// rows [J, J + w) of every right-hand side: solve with the unit-lower (LOWER) or the upper
// diagonal block of the factors, staged in shared memory; one warp per right-hand side
template <bool LOWER>
__global__ void trsv_block_kernel(const RsLaunch a, int J, int warps, int W) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tri = reinterpret_cast<double2*>(smem_raw);  // kBlk x kBlk, column-major
  double2* dinv = tri + kBlk * kBlk;
  double2* cols = dinv + kBlk;
  const RsJob jb = a.jobs[blockIdx.x];
  const int n = jb.n;
  if (n > a.max_n || J >= n) return;  // uniform per block
  const int w = min(W, n - J);
  const double2* A = a.abase + jb.a_off + J + (long long)J * jb.lda;
  for (int e = threadIdx.x; e < kBlk * w; e += blockDim.x) {
    const int r = e % kBlk, q = e / kBlk;
    tri[e] = r < w ? A[r + (long long)q * jb.lda] : make_double2(0.0, 0.0);
  }
  if (!LOWER)
    for (int i = threadIdx.x; i < w; i += blockDim.x) dinv[i] = cinv(A[i + (long long)i * jb.lda]);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * warps + warp;
  if (c >= jb.nrhs) return;
  double2* b = a.bbase + jb.b_off + (long long)c * jb.ldb + J;
  double2* sb = cols + warp * kBlk;
  for (int i = lane; i < w; i += 32) sb[i] = b[i];
  __syncwarp();
  if (LOWER) {
    for (int k = 0; k < w; ++k) {
      const double2 bk = sb[k];
      for (int i = k + 1 + lane; i < w; i += 32) sb[i] = cfms(tri[i + k * kBlk], bk, sb[i]);
      __syncwarp();
    }
  } else {
    for (int k = w - 1; k >= 0; --k) {
      const double2 bk = cmul(sb[k], dinv[k]);
      __syncwarp();
      if (lane == 0) sb[k] = bk;
      for (int i = lane; i < k; i += 32) sb[i] = cfms(tri[i + k * kBlk], bk, sb[i]);
      __syncwarp();
    }
  }
  for (int i = lane; i < w; i += 32) b[i] = sb[i];
}

// The same diagonal-block solve with the right-hand sides on the lanes (many blocks, the lower
// levels): an FP64 instruction costs this GPU the same issue time however many of its lanes
// are active, and here every lane works in every step, where the row-per-lane kernel above
// leaves the lanes past the triangle idle.  One block of four warps per (matrix, 32 right-hand
// sides); step k updates the rows below (above) k, split over the warps by row mod 4.
constexpr int kRhsWarps = 4;

template <bool LOWER>
__global__ void __launch_bounds__(kRhsWarps * 32) trsv_rhs_kernel(const RsLaunch a, int J, int W) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tri = reinterpret_cast<double2*>(smem_raw);  // kBlk x kBlk, column-major
  double2* xs = tri + kBlk * kBlk;                       // kBlk x 32: row i, lane l at i * 32 + l
  double2* dinv = xs + kBlk * 32;                        // kBlk
  const RsJob jb = a.jobs[blockIdx.x];
  const int n = jb.n;
  if (n > a.max_n || J >= n) return;  // uniform per block
  const int w = min(W, n - J);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = blockIdx.y * 32;
  if (c0 >= jb.nrhs) return;  // uniform per block
  const double2* A = a.abase + jb.a_off + J + (long long)J * jb.lda;
  double2* B = a.bbase + jb.b_off + J;
  for (int e = tid; e < kBlk * w; e += kRhsWarps * 32) {
    const int r = e % kBlk, q = e / kBlk;
    tri[e] = r < w ? A[r + (long long)q * jb.lda] : make_double2(0.0, 0.0);
  }
  if (!LOWER)
    for (int i = tid; i < w; i += kRhsWarps * 32) dinv[i] = cinv(A[i + (long long)i * jb.lda]);
  // the 32 right-hand sides' rows of the block (reads along columns)
  for (int e = tid; e < w * 32; e += kRhsWarps * 32) {
    const int i = e % w, cl = e / w, col = c0 + cl;
    xs[i * 32 + cl] = col < jb.nrhs ? B[i + (long long)col * jb.ldb] : make_double2(0.0, 0.0);
  }
  if (LOWER) {
    for (int k = 0; k < w; ++k) {
      __syncthreads();  // row k is final
      const double2 xk = xs[k * 32 + lane];
      for (int i = k + 1 + ((warp - (k + 1)) & (kRhsWarps - 1)); i < w; i += kRhsWarps)
        xs[i * 32 + lane] = cfms(tri[i + k * kBlk], xk, xs[i * 32 + lane]);
    }
  } else {
    for (int k = w - 1; k >= 0; --k) {
      __syncthreads();  // row k is final up to its diagonal
      const double2 xk = cmul(xs[k * 32 + lane], dinv[k]);
      __syncthreads();  // every warp has read row k before its owner rewrites it
      if ((k & (kRhsWarps - 1)) == warp) xs[k * 32 + lane] = xk;
      const int d = (k - warp) & (kRhsWarps - 1);  // the own rows below k: k - d, k - d - 4, ...
      for (int i = k - (d ? d : kRhsWarps); i >= 0; i -= kRhsWarps)
        xs[i * 32 + lane] = cfms(tri[i + k * kBlk], xk, xs[i * 32 + lane]);
    }
  }
  __syncthreads();
  for (int e = tid; e < w * 32; e += kRhsWarps * 32) {
    const int i = e % w, cl = e / w, col = c0 + cl;
    if (col < jb.nrhs) B[i + (long long)col * jb.ldb] = xs[i * 32 + cl];
  }
}

// The whole solve of a block of at most kBlk rows with the right-hand sides on the lanes
// (the many small k x k blocks of Atilde at the lower levels): x = P b, then the unit lower
// and the upper solve, in shared memory, four warps splitting the rows of each step.
__global__ void __launch_bounds__(kRhsWarps * 32) getrs_rhs_small_kernel(const RsLaunch a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tri = reinterpret_cast<double2*>(smem_raw);  // kBlk x kBlk, column-major (the LU factors)
  double2* xs = tri + kBlk * kBlk;                       // kBlk x 32
  double2* dinv = xs + kBlk * 32;                        // kBlk
  int* perm = reinterpret_cast<int*>(dinv + kBlk);       // kBlk
  const RsJob jb = a.jobs[blockIdx.x];
  const int n = jb.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = blockIdx.y * 32;
  if (n > kBlk || n > a.max_n || n <= 0 || c0 >= jb.nrhs) return;  // uniform per block
  const double2* A = a.abase + jb.a_off;
  double2* B = a.bbase + jb.b_off;
  load_perm(perm, a, jb, n);
  for (int e = tid; e < kBlk * n; e += kRhsWarps * 32) {
    const int r = e % kBlk, q = e / kBlk;
    tri[e] = r < n ? A[r + (long long)q * jb.lda] : make_double2(0.0, 0.0);
  }
  for (int i = tid; i < n; i += kRhsWarps * 32) dinv[i] = cinv(A[i + (long long)i * jb.lda]);
  __syncthreads();
  for (int e = tid; e < n * 32; e += kRhsWarps * 32) {
    const int i = e % n, cl = e / n, col = c0 + cl;
    xs[i * 32 + cl] = col < jb.nrhs ? B[perm[i] + (long long)col * jb.ldb] : make_double2(0.0, 0.0);
  }
  for (int k = 0; k < n; ++k) {  // unit lower
    __syncthreads();
    const double2 xk = xs[k * 32 + lane];
    for (int i = k + 1 + ((warp - (k + 1)) & (kRhsWarps - 1)); i < n; i += kRhsWarps)
      xs[i * 32 + lane] = cfms(tri[i + k * kBlk], xk, xs[i * 32 + lane]);
  }
  for (int k = n - 1; k >= 0; --k) {  // upper
    __syncthreads();
    const double2 xk = cmul(xs[k * 32 + lane], dinv[k]);
    __syncthreads();
    if ((k & (kRhsWarps - 1)) == warp) xs[k * 32 + lane] = xk;
    const int d = (k - warp) & (kRhsWarps - 1);
    for (int i = k - (d ? d : kRhsWarps); i >= 0; i -= kRhsWarps)
      xs[i * 32 + lane] = cfms(tri[i + k * kBlk], xk, xs[i * 32 + lane]);
  }
  __syncthreads();
  for (int e = tid; e < n * 32; e += kRhsWarps * 32) {
    const int i = e % n, cl = e / n, col = c0 + cl;
    if (col < jb.nrhs) B[i + (long long)col * jb.ldb] = xs[i * 32 + cl];
  }
}

// Inverses of the 64-row diagonal blocks of the factors, for the blocked solve that applies
// them on the tensor cores: block (matrix blockIdx.x, row block blockIdx.y), side blockIdx.z / 8
// (0: L's unit-lower block, 1: U's upper block), columns 8 (blockIdx.z % 8) .. + 7 of the
// inverse.  Column c of the inverse solves the block against e_c by substitution, the eight
// columns on lanes (lane % 8) and the rows on 16 slots (warp, lane / 8), four rows each; one
// block barrier per step publishes the step's value of each column.  Written to dinv: per
// (matrix, row block) the inverse of L's block then of U's block, 64 x 64 column-major (entries
// outside the block's w x w are zero).
constexpr int kInvThreads = 128;
__global__ void __launch_bounds__(kInvThreads) trinv_kernel(const RsLaunch a, int nbmax) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tri = reinterpret_cast<double2*>(smem_raw);  // 64 x 64, column-major: tri[k * 64 + i]
  double2* dinv_u = tri + 64 * 64;                      // 1 / U_kk
  double2* xs = dinv_u + 64;                             // [2][8]: the step's values, by parity
  const RsJob jb = a.jobs[blockIdx.x];
  const int J = blockIdx.y * 64;
  const int n = jb.n;
  if (n > a.max_n || J >= n) return;  // uniform per block
  const int w = min(64, n - J);
  const int upper = blockIdx.z >> 3, g = blockIdx.z & 7;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cl = lane & 7, slot = warp * 4 + (lane >> 3);
  const int col = 8 * g + cl;
  const double2* A = a.abase + jb.a_off + J + (long long)J * jb.lda;
  // the columns the steps below read: k >= 8g (L side), k <= 8g + 7 (U side)
  const int klo = upper ? 0 : 8 * g, khi = upper ? min(8 * g + 8, w) : w;
  for (int e = tid + klo * 64; e < khi * 64; e += kInvThreads) {
    const int i = e & 63, k = e >> 6;
    tri[e] = i < w ? A[i + (long long)k * jb.lda] : make_double2(0.0, 0.0);
  }
  if (upper)
    for (int k = tid; k < w; k += kInvThreads) dinv_u[k] = cinv(A[k + (long long)k * jb.lda]);
  double2 x[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) x[m] = make_double2(slot + 16 * m == col && col < w ? 1.0 : 0.0, 0.0);
  __syncthreads();
  int par = 0;
  if (!upper) {
    // L y = e_col: for k = 8g .. w - 2, rows i > k take -L_ik y_k (y_k = 0 for k < col)
#pragma unroll
    for (int mk = 0; mk < 4; ++mk) {
      for (int kk = 0; kk < 16; ++kk) {
        const int k = 16 * mk + kk;
        if (k < 8 * g || k >= w - 1) continue;  // uniform
        if (slot == kk) xs[par * 8 + cl] = x[mk];
        __syncthreads();
        const double2 xk = xs[par * 8 + cl];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          if (16 * m + 15 <= k) continue;  // uniform: no row of this layer below k
          const int i = slot + 16 * m;
          if (i > k && i < w) x[m] = cfms(tri[k * 64 + i], xk, x[m]);
        }
        par ^= 1;
      }
    }
  } else {
    // U y = e_col: for k = min(8g + 7, w - 1) .. 0, y_k /= U_kk, rows i < k take -U_ik y_k
    const int kmax = min(8 * g + 7, w - 1);
#pragma unroll
    for (int mk = 3; mk >= 0; --mk) {
      for (int kk = 15; kk >= 0; --kk) {
        const int k = 16 * mk + kk;
        if (k > kmax) continue;  // uniform
        if (slot == kk) {
          x[mk] = cmul(x[mk], dinv_u[k]);
          xs[par * 8 + cl] = x[mk];
        }
        __syncthreads();
        const double2 xk = xs[par * 8 + cl];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          if (16 * m >= k) continue;  // uniform: no row of this layer above k
          const int i = slot + 16 * m;
          if (i < k) x[m] = cfms(tri[k * 64 + i], xk, x[m]);
        }
        par ^= 1;
      }
    }
  }
  double2* out = a.dinv + (((long long)blockIdx.x * nbmax + blockIdx.y) * 2 + upper) * 4096 + (long long)col * 64;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int i = slot + 16 * m;
    out[i] = (i < w && col < w) ? x[m] : make_double2(0.0, 0.0);
  }
}

cudaError_t getrs_blocked_tc(const RsLaunch& a, cudaStream_t s) {
  const int max_n = a.max_n;
  int warps = kRsMaxWarps;
  while (warps > 2 && (long long)a.njobs * ((a.max_rhs + warps - 1) / warps) < 2 * device_sm_count()) warps /= 2;
  size_t psmem = 0;
  for (;; warps /= 2) {
    psmem = (size_t)max_n * sizeof(double2) * warps + (size_t)max_n * sizeof(int);
    if (psmem <= 200 * 1024 || warps == 1) break;
  }
  if (psmem > 200 * 1024) return cudaErrorInvalidValue;
  const size_t tsmem = (size_t)(kBlk * kBlk + kBlk + warps * kBlk) * sizeof(double2);
  // many blocks: the diagonal solves with the right-hand sides on the lanes
  const bool rhs_lanes = a.njobs >= 32;
  const size_t rsmem = (size_t)(kBlk * kBlk + kBlk * 32 + kBlk) * sizeof(double2);
  const dim3 rgrid(a.njobs, (a.max_rhs + 31) / 32);
  cudaError_t e = cudaFuncSetAttribute(permute_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(trsv_block_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(trsv_block_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
  if (e == cudaSuccess && rhs_lanes)
    e = cudaFuncSetAttribute(trsv_rhs_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
  if (e == cudaSuccess && rhs_lanes)
    e = cudaFuncSetAttribute(trsv_rhs_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
  if (e != cudaSuccess) return e;
  const dim3 grid(a.njobs, (a.max_rhs + warps - 1) / warps);
  permute_kernel<<<grid, warps * 32, psmem, s>>>(a, warps);
  symhss::count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ZgemmLaunch g;
  g.A = a.abase; g.B = a.bbase; g.C = a.bbase;
  g.jobs = nullptr; g.tiles = nullptr;
  g.mode = ZGEMM_SUB;
  g.status = a.status;
  g.wait_ns = 0;
  g.rs_jobs = a.jobs;
  g.njobs = a.njobs;
  g.img = a.zimg;
  g.img_bytes = a.zimg_bytes;
  g.ntiles_c = (a.max_rhs + zgemm_tc_tile_cols() - 1) / zgemm_tc_tile_cols();
  // forward: L y = P b, block by block; the rows below a block are updated on the tensor cores
  const int W = (a.blk == 16 || a.blk == 32) ? a.blk : kBlk;
  g.block_w = W;
  // one serial chain on s: every kernel after the permutation is a programmatic dependent of
  // the one before it
  g.chained = 1;
  // with the inverse scratch: the diagonal blocks through their inverses, formed once
  // (trinv_kernel) and applied as tensor-core products, instead of substitutions on the FP64
  // pipe (one right-hand side per warp for few matrices, per lane for many)
  const int nbmax = (max_n + 63) / 64;
  if (W == kBlk && a.dinv && a.dinv_bytes >= getrs_dinv_bytes(a.njobs, max_n)) {
    const size_t ismem = (size_t)(64 * 64 + 64 + 16) * sizeof(double2);
    if ((e = cudaFuncSetAttribute(trinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem)) !=
        cudaSuccess)
      return e;
    e = launch_chained(true, trinv_kernel, dim3(a.njobs, nbmax, 16), dim3(kInvThreads), ismem, s, a, nbmax);
    symhss::count_launches(1);
    if (e != cudaSuccess) return e;
    ZgemmLaunch gd = g;
    gd.A = a.dinv;
    gd.mode = ZGEMM_SET;
    gd.inv_nb = nbmax;
    gd.mtiles = 1;  // a 64-row block
    gd.ntiles = a.njobs * gd.ntiles_c;
    for (int J = 0; J < max_n; J += W) {
      gd.derive = ZGEMM_RS_FWD_DIAG;
      gd.block_j = J;
      if ((e = launch_zgemm_tc(gd, s)) != cudaSuccess) return e;
      const int below = max_n - J - W;
      if (below > 0) {
        g.derive = ZGEMM_RS_FWD;
        g.block_j = J;
        g.mtiles = (below + zgemm_tc_tile_rows() - 1) / zgemm_tc_tile_rows();
        g.ntiles = a.njobs * g.mtiles * g.ntiles_c;
        if ((e = launch_zgemm_tc(g, s)) != cudaSuccess) return e;
      }
    }
    for (int J = ((max_n - 1) / W) * W; J >= 0; J -= W) {
      gd.derive = ZGEMM_RS_BWD_DIAG;
      gd.block_j = J;
      if ((e = launch_zgemm_tc(gd, s)) != cudaSuccess) return e;
      if (J > 0) {
        g.derive = ZGEMM_RS_BWD;
        g.block_j = J;
        g.mtiles = (J + zgemm_tc_tile_rows() - 1) / zgemm_tc_tile_rows();
        g.ntiles = a.njobs * g.mtiles * g.ntiles_c;
        if ((e = launch_zgemm_tc(g, s)) != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  }
  for (int J = 0; J < max_n; J += W) {
    if (rhs_lanes) e = launch_chained(true, trsv_rhs_kernel<true>, rgrid, dim3(kRhsWarps * 32), rsmem, s, a, J, W);
    else e = launch_chained(true, trsv_block_kernel<true>, grid, dim3(warps * 32), tsmem, s, a, J, warps, W);
    symhss::count_launches(1);
    if (e != cudaSuccess) return e;
    const int below = max_n - J - W;
    if (below > 0) {
      g.derive = ZGEMM_RS_FWD;
      g.block_j = J;
      g.mtiles = (below + zgemm_tc_tile_rows() - 1) / zgemm_tc_tile_rows();
      g.ntiles = a.njobs * g.mtiles * g.ntiles_c;
      if ((e = launch_zgemm_tc(g, s)) != cudaSuccess) return e;
    }
  }
  // backward: U x = y from the last block; the rows above a block are updated on the tensor cores
  for (int J = ((max_n - 1) / W) * W; J >= 0; J -= W) {
    if (rhs_lanes) e = launch_chained(true, trsv_rhs_kernel<false>, rgrid, dim3(kRhsWarps * 32), rsmem, s, a, J, W);
    else e = launch_chained(true, trsv_block_kernel<false>, grid, dim3(warps * 32), tsmem, s, a, J, warps, W);
    symhss::count_launches(1);
    if (e != cudaSuccess) return e;
    if (J > 0) {
      g.derive = ZGEMM_RS_BWD;
      g.block_j = J;
      g.mtiles = (J + zgemm_tc_tile_rows() - 1) / zgemm_tc_tile_rows();
      g.ntiles = a.njobs * g.mtiles * g.ntiles_c;
      if ((e = launch_zgemm_tc(g, s)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace

template <typename CT>
cudaError_t getrs_impl(const RsLaunch& a, cudaStream_t s) {
  const int max_n = a.max_n;
  if (a.njobs <= 0 || a.max_rhs <= 0) return cudaSuccess;
  cudaError_t e;
  // FP64 with many right-hand sides and blocks larger than one diagonal block: blocked solve
  // whose off-diagonal updates run on the tensor cores
  // lu_tc = 2: the blocked tensor-core solve for many blocks or many right-hand sides in total
  // (its block updates then fill the product's tiles), the unblocked FP64 solve otherwise
  const bool use_tc = (a.tc == 1 || (a.tc == 2 && (a.njobs >= 32 || (long long)a.njobs * a.max_rhs >= 512))) &&
                      a.zimg && a.zimg_bytes >= zgemm_rs_img_bytes(a.njobs, a.max_n, a.max_rhs);
  if (sizeof(CT) == sizeof(double2) && use_tc && a.status && a.max_rhs > 4 &&
      max_n > ((a.blk == 16 || a.blk == 32) ? a.blk : kBlk))
    return getrs_blocked_tc(a, s);
  if (sizeof(CT) == sizeof(double2) && a.max_rhs > 4 && max_n <= kBlk && a.njobs >= 32) {
    // many small blocks: the whole solve with the right-hand sides on the lanes
    const size_t smem = (size_t)(kBlk * kBlk + kBlk * 32 + kBlk) * sizeof(double2) + kBlk * sizeof(int);
    e = cudaFuncSetAttribute(getrs_rhs_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    getrs_rhs_small_kernel<<<dim3(a.njobs, (a.max_rhs + 31) / 32), kRhsWarps * 32, smem, s>>>(a);
    symhss::count_launches(1);
    return cudaGetLastError();
  }
  if (a.max_rhs <= 4 && sizeof(CT) == sizeof(double2) && max_n >= 128) {
    // few large blocks: a cluster per (matrix, right-hand side) while the SMs allow
    const int nb = (max_n + 31) / 32;
    int C = 16;
    while (C >= 2 && ((long long)a.njobs * a.max_rhs * C > device_sm_count() || nb < C)) C /= 2;
    if (C >= 2) {
      const int nbown = (nb + C - 1) / C;
      const size_t smem = (size_t)max_n * sizeof(double2) + (size_t)nbown * (1024 + 32 + 512) * sizeof(double2) +
                          (size_t)max_n * sizeof(int);
      if (smem <= 200 * 1024) {
        e = cudaFuncSetAttribute(getrs_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess && C > 8)
          e = cudaFuncSetAttribute(getrs_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(a.njobs * a.max_rhs * C, 1, 1);
        cfg.blockDim = dim3(kClThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, getrs_cluster_kernel, a, nbown);
        symhss::count_launches(1);
        return e;
      }
    }
  }
  if (a.max_rhs <= 4) {
    const size_t smem = (size_t)max_n * (2 * sizeof(CT) + sizeof(int));
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(getrs_cta_kernel<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    getrs_cta_kernel<CT><<<dim3(a.njobs, a.max_rhs), kCtaThreads, smem, s>>>(a);
    symhss::count_launches(1);
    return cudaGetLastError();
  }
  // fewer warps per block when the batch is small (top levels: few boxes, many right-hand
  // sides), so that the grid covers every SM twice: each SM's FP64 pipe bounds its warps
  int warps = kRsMaxWarps;
  while (warps > 2 && (long long)a.njobs * ((a.max_rhs + warps - 1) / warps) < 2 * device_sm_count()) warps /= 2;
  size_t smem = 0;
  for (;; warps /= 2) {
    smem = (size_t)max_n * sizeof(CT) * (1 + warps) + (size_t)max_n * sizeof(int);
    if (smem <= 200 * 1024 || warps == 1) break;
  }
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(getrs_kernel<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.njobs, (a.max_rhs + warps - 1) / warps);
  getrs_kernel<CT><<<grid, warps * 32, smem, s>>>(a, warps);
  symhss::count_launches(1);
  return cudaGetLastError();
}

long long getrs_dinv_bytes(int njobs, int max_n) {
  return (long long)njobs * ((max_n + 63) / 64) * 2 * 4096 * (long long)sizeof(double2);
}

cudaError_t launch_getrs(const RsLaunch& a, cudaStream_t s) {
  return a.abase32 ? getrs_impl<float2>(a, s) : getrs_impl<double2>(a, s);
}

}  // namespace symhss
