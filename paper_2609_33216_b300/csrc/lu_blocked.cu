// Batched blocked LU with partial pivoting (the diagonal-block factorisations of
// Sec. 4.2), right-looking with panel width kNb.  All matrices of a batch advance
// panel by panel in lock step; every panel step is three launches whose work
// spreads over many thread blocks even when the batch holds a single matrix (the
// root block):
//   1. panel: one block per matrix factors columns [j, j + w) of rows [j, n) with
//      partial pivoting (swaps applied inside the panel only), the panel held in
//      shared memory when it fits;
//   2. swaps + TRSM: one warp per column outside the panel applies the panel's
//      row interchanges and, right of the panel, solves L11 U12 = A12;
//   3. trailing update: A22 -= L21 U12 in 32 x 32 tiles, one block per tile.
// The pivots follow the LAPACK convention (row ipiv[k] was swapped with row k at
// step k), so the result is interchangeable with the unblocked factorisation.
#include <algorithm>

#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace symhss {

namespace {

constexpr int kNb = 16;          // panel width
constexpr int kOuterMax = 64;    // largest column block of the tensor-core trailing update (FP64)
constexpr int kTcMinJobs = 32;   // lu_tc = 2: the tensor-core path for launches of this many matrices
constexpr int kPanelThreads = 256;
constexpr int kPanelWarps = kPanelThreads / 32;
constexpr int kTs = 32;          // trailing-update tile
constexpr int kClusterPanelThreads = 256;

struct CandK { long long k; int i; };

template <typename CT> __device__ __forceinline__ CT* lu_base(const LuLaunch& a);
template <> __device__ __forceinline__ double2* lu_base<double2>(const LuLaunch& a) { return a.base; }
template <> __device__ __forceinline__ float2* lu_base<float2>(const LuLaunch& a) { return a.base32; }

template <typename CT>
__global__ void __launch_bounds__(kPanelThreads) panel_kernel(const LuLaunch a, int j) {
  __shared__ long long redk[kPanelWarps];
  __shared__ int redi[kPanelWarps];
  __shared__ int s_piv, s_zero;
  __shared__ CT s_row[kNb];
  __shared__ CT s_inv;
  const LuJob jb = a.jobs[blockIdx.x];
  const int n = jb.n, ld = jb.ld;
  if (j >= n) return;
  const int w = min(kNb, n - j);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  CT* A = lu_base<CT>(a) + jb.a_off;
  int* piv = a.piv + jb.piv_off;
  for (int c = 0; c < w; ++c) {
    const int jc = j + c;
    const CT* col = A + (long long)jc * ld;
    long long bk = -1;
    int bi = n;
    for (int i = jc + tid; i < n; i += kPanelThreads) {
      const long long k = pivot_key(cabs1(col[i]));
      if (k > bk || (k == bk && i < bi)) { bk = k; bi = i; }
    }
    warp_argmax_key(bk, bi);
    if (lane == 0) { redk[warp] = bk; redi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      bk = lane < kPanelWarps ? redk[lane] : -1;
      bi = lane < kPanelWarps ? redi[lane] : n;
      warp_argmax_key(bk, bi);
      if (lane == 0) {
        // an exactly zero (or no finite) pivot skips the step; every barrier stays unconditional
        const bool zero = bk <= 0 || bi >= n;
        s_piv = zero ? jc : bi;
        s_zero = zero;
        piv[jc] = s_piv;
        if (zero) {
          if (a.info[jb.info_idx] == 0) a.info[jb.info_idx] = jc + 1;
          atomicOr(a.status, ST_SINGULAR);
        }
      }
    }
    __syncthreads();
    const int p = s_piv;
    const bool zero = s_zero;
    if (!zero && tid < w && p != jc) {
      CT* cc = A + (long long)(j + tid) * ld;
      const CT t = cc[jc];
      cc[jc] = cc[p];
      cc[p] = t;
    }
    __syncthreads();
    if (tid < w) {
      const CT v = A[jc + (long long)(j + tid) * ld];
      s_row[tid] = v;
      if (tid == c) s_inv = zero ? make_c<CT>(0.0, 0.0) : cinv_pivot(v);
    }
    __syncthreads();
    const CT inv = s_inv;
    for (int i = jc + 1 + tid; !zero && i < n; i += kPanelThreads) {
      const CT l = cmul(A[i + (long long)jc * ld], inv);
      A[i + (long long)jc * ld] = l;
      for (int q = c + 1; q < w; ++q) {
        CT* cq = A + (long long)(j + q) * ld;
        cq[i] = cfms(l, s_row[q], cq[i]);
      }
    }
    __syncthreads();
  }
}

// Panel factorisation with the panel (rows [j, n) x w columns) staged in shared
// memory; the pivot search of column c + 1 is fused into the update of column c.
// THREADS is chosen per launch so that each thread holds about one or two panel rows.
// FP64 issues slowly on this GPU, so only the row updates use it: the pivot search
// compares integer keys and one thread forms the pivot's reciprocal for the block.
template <int THREADS, typename CT>
__global__ void __launch_bounds__(THREADS) panel_smem_kernel(const LuLaunch a, int j) {
  constexpr int kWarps = THREADS / 32;
  extern __shared__ __align__(16) unsigned char p_raw[];
  CT* P = reinterpret_cast<CT*>(p_raw);  // column-major: P[q * rows + i]
  __shared__ long long redk[kWarps];
  __shared__ int redi[kWarps];
  __shared__ int s_piv, s_zero;
  __shared__ CT s_inv;
  const LuJob jb = a.jobs[blockIdx.x];
  const int n = jb.n, ld = jb.ld;
  if (j >= n) return;  // uniform per block
  const int w = min(kNb, n - j), rows = n - j;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  CT* A = lu_base<CT>(a) + jb.a_off;
  int* piv = a.piv + jb.piv_off;
  for (int e = tid; e < rows * w; e += THREADS) {
    const int i = e % rows, q = e / rows;
    P[q * rows + i] = A[j + i + (long long)(j + q) * ld];
  }
  __syncthreads();
  long long bk = -1;
  int bi = rows;
  for (int i = tid; i < rows; i += THREADS) {
    const long long k = pivot_key(cabs1(P[i]));
    if (k > bk || (k == bk && i < bi)) { bk = k; bi = i; }
  }
  for (int c = 0; c < w; ++c) {
    warp_argmax_key(bk, bi);
    if (lane == 0) { redk[warp] = bk; redi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      bk = lane < kWarps ? redk[lane] : -1;
      bi = lane < kWarps ? redi[lane] : rows;
      warp_argmax_key(bk, bi);
      if (lane == 0) {
        // an exactly zero (or no finite) pivot skips the step; every barrier stays unconditional
        const bool zero = bk <= 0 || bi >= rows;
        const int p = zero ? c : bi;
        s_piv = p;
        s_zero = zero;
        s_inv = zero ? make_c<CT>(0.0, 0.0) : cinv_pivot(P[c * rows + p]);
        piv[j + c] = j + p;
        if (zero) {
          if (a.info[jb.info_idx] == 0) a.info[jb.info_idx] = j + c + 1;
          atomicOr(a.status, ST_SINGULAR);
        }
      }
    }
    __syncthreads();
    const int p = s_piv;
    const bool zero = s_zero;
    if (!zero && tid < w && p != c) {
      const CT t = P[tid * rows + c];
      P[tid * rows + c] = P[tid * rows + p];
      P[tid * rows + p] = t;
    }
    __syncthreads();
    const CT inv = s_inv;
    bk = -1;
    bi = rows;
    for (int i = c + 1 + tid; i < rows; i += THREADS) {
      if (!zero) {
        const CT l = cmul(P[c * rows + i], inv);
        P[c * rows + i] = l;
        for (int q = c + 1; q < w; ++q) P[q * rows + i] = cfms(l, P[q * rows + c], P[q * rows + i]);
      }
      if (c + 1 < w) {
        const long long k = pivot_key(cabs1(P[(c + 1) * rows + i]));
        if (k > bk || (k == bk && i < bi)) { bk = k; bi = i; }
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < rows * w; e += THREADS) {
    const int i = e % rows, q = e / rows;
    A[j + i + (long long)(j + q) * ld] = P[q * rows + i];
  }
}


// Panel factorisation by a thread-block cluster of C blocks (one cluster per matrix), for
// the few large matrices of the top levels whose panel would otherwise run on one SM.
// Panel row i (rows [j, n) numbered from 0) lives in block i % C at local index i / C, in
// shared memory, and never moves: the interchanges are kept as a permutation (pos2phys /
// phys2pos, the same in every block) and applied when the panel is written back.  Column
// step c: every block publishes its candidate -- the largest |re| + |im| key among its rows
// not yet pivoted, ties to the lowest current position (the one-block kernel's pivots) --
// together with that row's w entries; after ONE cluster barrier every block reads the C keys
// through distributed shared memory, takes the largest, copies the winner's row from the
// winner's candidate slot, updates the permutation, and updates its own unpivoted rows
// (fusing the next column's candidate).  A pivot row is no longer written once chosen, and a
// candidate slot is double-buffered, so no second barrier is needed.  The arithmetic of every
// row is the one-block kernel's, so the factors are identical.
struct CandRow {
  long long k;
  int pos, phys;
  double2 row[kNb];
};

__global__ void __launch_bounds__(kClusterPanelThreads) panel_cluster_kernel(const LuLaunch a, int j, int lmax) {
  pdl_enter();
  extern __shared__ __align__(16) double2 P[];  // P[q * lmax + li]; then pos2phys, phys2pos
  constexpr int kWarps = kClusterPanelThreads / 32;
  __shared__ long long redk[kWarps];
  __shared__ int redi[kWarps], redr[kWarps];
  __shared__ CandRow cand[2];
  __shared__ int s_zero[2];
  __shared__ double2 prow[2][kNb];  // pivot rows of the last two columns (by column parity)
  __shared__ double2 s_inv;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int lgC = __ffs(C) - 1;  // C is a power of two
  const int rank = (int)cl.block_rank();
  const LuJob jb = a.jobs[blockIdx.x / C];
  const int n = jb.n, ld = jb.ld;
  if (j >= n) return;  // uniform over the cluster (one matrix per cluster)
  const int w = min(kNb, n - j), rows = n - j;
  const int lrows = rank < rows ? (rows - rank + C - 1) / C : 0;
  if ((rows + C - 1) / C > lmax || rows > a.max_n) {  // uniform over the cluster
    if (threadIdx.x == 0 && rank == 0) atomicOr(a.status, ST_BAD_INDEX);
    return;
  }
  int* pos2phys = reinterpret_cast<int*>(P + (size_t)kNb * lmax);
  int* phys2pos = pos2phys + a.max_n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double2* A = a.base + jb.a_off;
  int* piv = a.piv + jb.piv_off;
  for (int e = tid; e < lrows * w; e += kClusterPanelThreads) {
    const int li = e % lrows, q = e / lrows;
    P[q * lmax + li] = A[j + rank + li * C + (long long)(j + q) * ld];
  }
  for (int i = tid; i < rows; i += kClusterPanelThreads) { pos2phys[i] = i; phys2pos[i] = i; }
  __syncthreads();
  // candidate for column 0: (key, current position, physical row)
  long long bk = -1;
  int bi = rows, br = -1;
  for (int li = tid; li < lrows; li += kClusterPanelThreads) {
    const int r = rank + li * C;
    const long long k = pivot_key(cabs1(P[li]));
    if (k > bk || (k == bk && r < bi)) { bk = k; bi = r; br = r; }
  }
  // Column c: the block's candidate row and the cluster's choice need column c updated for
  // every earlier pivot, but the other columns of the rank-1 update of pivot c - 1 (c + 1 ..
  // w - 1) wait: warps 1 .. 7 apply them between their arrival at the cluster barrier of
  // column c and their wait, while warp 0 waits and picks the pivot, so the update is off the
  // serial path.  The one row that cannot wait, the block's candidate (its entries go to every
  // block of the cluster), warp 0 updates on its own before publishing it.
  int par = 0;
  for (int c = 0; c < w; ++c) {
    const bool lag = c >= 1 && !s_zero[(c - 1) & 1];  // pivot c - 1's update of columns > c is pending
    // block's best (ties: lowest position), then publish it with its row
    warp_argmax_key_redux(bk, bi, br);
    if (lane == 0) { redk[warp] = bk; redi[warp] = bi; redr[warp] = br; }
    __syncthreads();
    if (warp == 0) {
      bk = lane < kWarps ? redk[lane] : -1;
      bi = lane < kWarps ? redi[lane] : rows;
      br = lane < kWarps ? redr[lane] : -1;
      warp_argmax_key_redux(bk, bi, br);
      if (lane == 0) { cand[par].k = bk; cand[par].pos = bi; cand[par].phys = br; }
      const int li = br >= 0 ? (br - rank) >> lgC : 0;
      if (lane < w) {
        double2 v = br >= 0 ? P[lane * lmax + li] : make_double2(0.0, 0.0);
        // the pending update of pivot c - 1 on this row (the same arithmetic the deferred
        // update below applies to it)
        if (br >= 0 && lag && lane > c) v = cfms(P[(c - 1) * lmax + li], prow[(c - 1) & 1][lane], v);
        cand[par].row[lane] = v;
      }
    }
    __syncthreads();  // the candidate row is read before the deferred update writes it
    asm volatile("barrier.cluster.arrive.release;" ::: "memory");
    if (warp == 0) {
      asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
      // the C proposals (one lane each) with their pivot entries, whose reciprocals are
      // formed while the shuffles pick the winner; the winner's row; the interchange of
      // positions c and p in the permutation
      long long ck = -1;
      int cp = rows, cb = -1;
      double2 pv = make_double2(0.0, 0.0);
      if (lane < C) {
        const CandRow* cd = cl.map_shared_rank(&cand[par], lane);
        ck = cd->k;
        cp = cd->pos;
        pv = cd->row[c];
        cb = lane;
      }
      const double2 pinv = lane < C ? cinv_pivot(pv) : make_double2(0.0, 0.0);
      warp_argmax_key_redux(ck, cp, cb);
      const bool zero = ck <= 0 || cp >= rows || cb < 0;
      const int p = zero ? c : cp;  // current position of the pivot row
      const double ix = __shfl_sync(0xffffffffu, pinv.x, cb < 0 ? 0 : cb);
      const double iy = __shfl_sync(0xffffffffu, pinv.y, cb < 0 ? 0 : cb);
      if (lane < w) prow[c & 1][lane] = zero ? make_double2(0.0, 0.0) : cl.map_shared_rank(&cand[par], cb)->row[lane];
      if (lane == 0) {
        s_inv = zero ? make_double2(0.0, 0.0) : make_double2(ix, iy);
        s_zero[c & 1] = zero;
        const int rc = pos2phys[c], rp = pos2phys[p];
        pos2phys[c] = rp; pos2phys[p] = rc;
        phys2pos[rp] = c; phys2pos[rc] = p;
        if (rank == 0) {
          piv[j + c] = j + p;
          if (zero) {
            if (a.info[jb.info_idx] == 0) a.info[jb.info_idx] = j + c + 1;
            atomicOr(a.status, ST_SINGULAR);
          }
        }
      }
    } else {
      if (lag) {
        // the deferred update of pivot c - 1, columns c + 1 .. w - 1 of the rows below it.
        // Warp 0 meanwhile swaps two positions >= c in phys2pos: either value of such a row
        // passes the test below, so the read needs no ordering.
        const int nq = w - c - 1;
        const double2* pr = prow[(c - 1) & 1];
        for (int e = tid - 32; e < lrows * nq; e += kClusterPanelThreads - 32) {
          const int li = e % lrows, q = c + 1 + e / lrows;
          if (phys2pos[rank + li * C] <= c - 1) continue;
          P[q * lmax + li] = cfms(P[(c - 1) * lmax + li], pr[q], P[q * lmax + li]);
        }
      }
      asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
    }
    par ^= 1;
    __syncthreads();
    const bool zero = s_zero[c & 1];
    const double2 inv = s_inv;
    // per own row not yet pivoted (current position > c), one thread: its multiplier, then the
    // rank-1 update of its column c + 1 alone (the next candidate; the rest waits, see above);
    // the arithmetic of each element is the one-block kernel's
    bk = -1;
    bi = rows;
    br = -1;
    for (int li = tid; li < lrows; li += kClusterPanelThreads) {
      const int r = rank + li * C;
      const int pos = phys2pos[r];
      if (pos <= c) continue;
      double2 l = P[c * lmax + li];
      if (!zero) {
        l = cmul(l, inv);
        P[c * lmax + li] = l;
      }
      if (c + 1 < w) {
        double2 v = P[(c + 1) * lmax + li];
        if (!zero) {
          v = cfms(l, prow[c & 1][c + 1], v);
          P[(c + 1) * lmax + li] = v;
        }
        const long long k = pivot_key(cabs1(v));
        if (k > bk || (k == bk && pos < bi)) { bk = k; bi = pos; br = r; }
      }
    }
  }
  cl.sync();  // no block reads another's candidate slots after this point
  for (int e = tid; e < lrows * w; e += kClusterPanelThreads) {
    const int li = e % lrows, q = e / lrows;
    const int r = rank + li * C;
    A[j + phys2pos[r] + (long long)(j + q) * ld] = P[q * lmax + li];
  }
}

// Row interchanges of a panel and, right of it, L11 U12 = A12, for 32 columns per block.
// The panel's w interchanges touch at most 2w rows; their composition is a
// permutation of that row set, built once per block, so each column is permuted by
// a single gather (lane l ends with the value of row rows[l]); rows j..j+w-1 of the 32
// columns then go through shared memory to the unit-lower 16 x 16 solve, which runs with
// one column per lane.
// tlo, thi: the solve covers only columns in [max(j + w, tlo), thi); swaps = 0: no
// interchanges (the columns are already permuted); cbase: first column of blockIdx.y = 0.
// CB columns per block: 32 (256 threads; the solve with the columns on the lanes and the rows
// over warps 0..3) or 8 (128 threads; the solve with lane = column + 8 x row group, each of the
// 16 rows on one thread: four times the blocks for the same FP64 work, for launches whose
// 32-column blocks would leave most SMs idle).
template <typename CT, int CB>
__global__ void __launch_bounds__(CB == 32 ? 256 : 128) swap_trsm_warp_kernel(const LuLaunch a, int j, int tlo,
                                                                               int thi, int swaps, int cbase) {
  constexpr int NT = CB == 32 ? 256 : 128, NW = NT / 32, CPW = CB / NW;
  pdl_enter();
  __shared__ CT l11[kNb][kNb];
  __shared__ int rows_s[2 * kNb];   // row set: j..j+w-1, then the outside pivot rows
  __shared__ int src_s[2 * kNb];    // lane l takes its new value from row src_s[l]
  __shared__ int nrows_s;
  const LuJob jb = a.jobs[blockIdx.x];
  const int n = jb.n, ld = jb.ld;
  if (j >= n) return;  // uniform per block
  const int w = min(kNb, n - j);
  CT* A = lu_base<CT>(a) + jb.a_off;
  __shared__ int piv_s[kNb];
  if (threadIdx.x < w) piv_s[threadIdx.x] = a.piv[jb.piv_off + j + threadIdx.x];
  for (int e = threadIdx.x; e < w * w; e += NT) {
    const int r = e % w, c = e / w;
    l11[r][c] = A[j + r + (long long)(j + c) * ld];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // warp 0, lane c for column c of the panel (a serial thread here cost more than the rest
    // of the kernel): the row set is rows j .. j + w - 1, then each pivot row outside them
    // once, in column order
    const unsigned full = 0xffffffffu;
    const int l = threadIdx.x;
    const int p = l < w ? piv_s[l] : -1;
    const unsigned same = __match_any_sync(full, p);
    const int lead = __ffs(same) - 1;  // lowest lane with the same pivot row
    const bool outside = l < w && p >= j + w;
    const unsigned fm = __ballot_sync(full, outside && lead == l);
    const int cnt = w + __popc(fm);
    if (outside && lead == l) rows_s[w + __popc(fm & ((1u << l) - 1))] = p;
    if (l < w) rows_s[l] = j + l;
    // position of column l's pivot row in the set (-1: none, which a valid pivot never gives)
    int lp = -1;
    if (l < w && p >= j) lp = p < j + w ? p - j : w + __popc(fm & ((1u << lead) - 1));
    __syncwarp();
    // content (lane l): the original row whose values end at rows_s[l]; the interchanges in order
    int content = l < cnt ? rows_s[l] : 0;
    for (int c = 0; swaps && c < w; ++c) {
      const int lpc = __shfl_sync(full, lp, c);
      if (lpc < 0 || lpc == c) continue;  // uniform
      const int vc = __shfl_sync(full, content, c);
      const int vp = __shfl_sync(full, content, lpc);
      if (l == c) content = vp;
      else if (l == lpc) content = vc;
    }
    if (l < cnt) src_s[l] = content;
    if (l == 0) nrows_s = cnt;
    // the same interchanges on the kept row permutation (once per panel: the first column block)
    if (swaps && a.perm && blockIdx.y == 0) {
      int* pm = a.perm + jb.piv_off;
      const int v = l < cnt ? pm[content] : 0;
      __syncwarp();
      if (l < cnt) pm[rows_s[l]] = v;
    }
  }
  __syncthreads();
  __shared__ CT xs[kNb][CB];  // rows j .. j + w - 1 of the block's CB columns, after the interchanges
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cnt = nrows_s;
  const int tl = max(j + w, tlo), th = min(thi, n);
  const int cfirst = cbase + blockIdx.y * CB;
  // a column takes part if it is interchanged, or (without interchanges) if it is solved
  auto part = [&](int col) {
    return col < n && !(col >= j && col < j + w) && (swaps || (col >= tl && col < th));
  };
  // interchanges: one column per warp at a time, the lanes over the row set
  // (the columns of a warp are loaded before any of them is written: each column's stores
  // touch only that column, so the loads need not wait for them)
  CT xv[CPW];
  const int src = lane < cnt ? src_s[lane] : 0;
#pragma unroll
  for (int i = 0; i < CPW; ++i) {
    const int col = cfirst + warp + NW * i;
    xv[i] = (part(col) && lane < cnt) ? A[(long long)col * ld + src] : make_c<CT>(0.0, 0.0);
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < CPW; ++i) {
    const int cl = warp + NW * i, col = cfirst + cl;
    if (!part(col)) continue;  // uniform per warp
    if (swaps && lane >= w && lane < cnt) A[(long long)col * ld + rows_s[lane]] = xv[i];
    if (lane < w) xs[lane][cl] = xv[i];
  }
  if (CB == 32) {
    // L11 U12 = A12 with the 32 columns on the lanes (every lane of an FP64 instruction works),
    // rows split over warps 0..3 by row mod 4
    const int col = cfirst + lane;
    const bool solve = col >= tl && col < th;
    for (int c = 0; c < w; ++c) {
      __syncthreads();  // row c is final
      if (warp < 4 && solve) {
        const CT xc = xs[c][lane % CB];
        for (int r = c + 1 + ((warp - (c + 1)) & 3); r < w; r += 4)
          xs[r][lane % CB] = cfms(l11[r][c], xc, xs[r][lane % CB]);
      }
    }
  } else {
    // column lane % 8, row warp + 4 (lane / 8): one row per thread, the four rows of a warp
    // in one instruction
    const int cl = lane & 7, r = warp + 4 * (lane >> 3);
    const int col = cfirst + cl;
    const bool solve = col >= tl && col < th && r < w;
    for (int c = 0; c < w; ++c) {
      __syncthreads();  // row c is final
      if (solve && r > c) xs[r][cl] = cfms(l11[r][c], xs[c][cl], xs[r][cl]);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < CB * w; e += NT) {
    const int r = e % w, cl = e / w;
    if (part(cfirst + cl)) A[(long long)(cfirst + cl) * ld + j + r] = xs[r][cl];
  }
}

// A22 -= L21 U12 for the tile (blockIdx.y, blockIdx.z) of every matrix, over the trailing
// columns [j + w + cskip, j + w + cskip + clen) (clen < 0: to the last column) and the
// trailing rows [j + w, j + w + rlen) (rlen < 0: to the last row)
template <typename CT>
__global__ void __launch_bounds__(256) update_kernel(const LuLaunch a, int j, int cskip, int clen, int rlen) {
  __shared__ CT at[kNb][kTs];      // L21 tile, transposed: at[c][r]
  __shared__ CT bt[kNb][kTs];      // U12 tile: bt[c][col]
  const LuJob jb = a.jobs[blockIdx.x];
  const int n0 = jb.n, ld = jb.ld;
  const int w = min(kNb, n0 - j);
  const int s = j + w;                   // first trailing row / column
  const int n = rlen < 0 ? n0 : min(n0, s + rlen);  // rows end here; columns at cend
  const int r0 = s + blockIdx.y * kTs, c0 = s + cskip + blockIdx.z * kTs;
  const int cend = clen < 0 ? n0 : min(n0, s + cskip + clen);
  if (j >= n0 || r0 >= n || c0 >= cend) return;
  CT* A = lu_base<CT>(a) + jb.a_off;
  const int tid = threadIdx.x;
  for (int e = tid; e < kNb * kTs; e += 256) {
    const int r = e % kTs, c = e / kTs;
    at[c][r] = (r0 + r < n && c < w) ? A[r0 + r + (long long)(j + c) * ld] : make_c<CT>(0.0, 0.0);
    const int cc = e % kNb, col = e / kNb;
    bt[cc][col] = (c0 + col < cend && cc < w) ? A[j + cc + (long long)(c0 + col) * ld] : make_c<CT>(0.0, 0.0);
  }
  __syncthreads();
  const int tx = tid & 31, ty = tid >> 5;  // row tx, columns ty + 8q
  const int row = r0 + tx;
  CT acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int col = c0 + ty + 8 * q;
    acc[q] = (row < n && col < cend) ? A[row + (long long)col * ld] : make_c<CT>(0.0, 0.0);
  }
#pragma unroll
  for (int c = 0; c < kNb; ++c) {
    const CT l = at[c][tx];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = cfms(l, bt[c][ty + 8 * q], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int col = c0 + ty + 8 * q;
    if (row < n && col < cend) A[row + (long long)col * ld] = acc[q];
  }
}

__global__ void zero_info_kernel(int* info, const LuJob* jobs, int njobs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < njobs) info[jobs[b].info_idx] = 0;
}

// the row permutation of every matrix starts as the identity (one block per matrix)
__global__ void perm_init_kernel(const LuLaunch a) {
  const LuJob jb = a.jobs[blockIdx.x];
  for (int i = threadIdx.x; i < jb.n; i += blockDim.x) a.perm[jb.piv_off + i] = i;
}

// Side stream (highest priority) and two events for the look-ahead, one set per host
// thread and device, created on first use; nullptr if they cannot be created (the
// factorisation then runs without look-ahead on the caller's stream).
struct LookAhead {
  cudaStream_t side = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
  bool failed = false;
};

LookAhead* look_ahead_streams() {
  constexpr int kMaxDev = 64;
  thread_local LookAhead per_dev[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return nullptr;
  }
  LookAhead& la = per_dev[dev];
  if (la.failed) return nullptr;
  if (!la.side) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&la.side, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&la.ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&la.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      la.failed = true;
      return nullptr;
    }
  }
  return &la;
}

}  // namespace

template <typename CT>
cudaError_t getrf_impl(const LuLaunch& a, cudaStream_t s) {
  if (a.njobs <= 0 || a.max_n <= 0) return cudaSuccess;
  zero_info_kernel<<<(a.njobs + 127) / 128, 128, 0, s>>>(a.info, a.jobs, a.njobs);
  symhss::count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.perm) {
    perm_init_kernel<<<a.njobs, 256, 0, s>>>(a);
    symhss::count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // panels of up to 780 rows fit in shared memory (780 x 16 x 16 B = 195 KB)
  const size_t panel_smem = (size_t)a.max_n * kNb * sizeof(CT);
  const bool smem_panel = panel_smem <= 200 * 1024;
  const int pcap = a.panel_threads >= 1024 ? 1024 : (a.panel_threads >= 512 ? 512 : 256);
  const int pthreads = std::min(pcap, a.max_n > 512 ? 1024 : (a.max_n > 256 ? 512 : 256));
  if (smem_panel) {
    // every variant the loop may pick as the panel shrinks
    e = cudaFuncSetAttribute(panel_smem_kernel<256, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem);
    if (e == cudaSuccess && pthreads >= 512)
      e = cudaFuncSetAttribute(panel_smem_kernel<512, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem);
    if (e == cudaSuccess && pthreads >= 1024)
      e = cudaFuncSetAttribute(panel_smem_kernel<1024, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem);
    if (e != cudaSuccess) return e;
  }
  const int ncolblk = (a.max_n + 31) / 32;  // 32 columns per block of the interchange kernel
  // 8 columns per block where 32-column blocks would leave most SMs idle (the upper levels)
  const int ncolblk8 = (a.max_n + 7) / 8;
  const bool narrow = (long long)a.njobs * ncolblk < device_sm_count();
  // Depth-1 look-ahead: after the interchanges and TRSM of panel j, the first trailing
  // tile column (which holds panel j + kNb) is updated first; panel j + kNb then runs on
  // a high-priority side stream while the rest of the trailing update runs on s.  The two
  // touch disjoint columns; s waits for the panel before the next interchanges.
  LookAhead* la = a.lookahead ? look_ahead_streams() : nullptr;
  // cluster panels for few large matrices: C blocks per matrix while the batch still leaves
  // SMs free and every block keeps at least 32 panel rows
  int pc = 1;
  while (sizeof(CT) == sizeof(double2) && pc < 16 && 2 * pc <= a.panel_cluster &&
         a.njobs * 2 * pc <= device_sm_count() && a.max_n / (2 * pc) >= 32)
    pc *= 2;
  const int lmax = (a.max_n + pc - 1) / pc;
  if (pc > 1) {
    e = cudaFuncSetAttribute(panel_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)lmax * kNb * sizeof(double2) + 2 * (size_t)a.max_n * sizeof(int)));
    if (e == cudaSuccess && pc > 8)
      e = cudaFuncSetAttribute(panel_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      pc = 1;
    }
  }
  // chained: a programmatic dependent launch of the kernel before it on the same stream (the
  // kernels of the tensor-core path's serial chain; each waits for its predecessor first)
  auto panel = [&](int jj, cudaStream_t st, bool chained) {
    if (pc > 1) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(a.njobs * pc, 1, 1);
      cfg.blockDim = dim3(kClusterPanelThreads, 1, 1);
      cfg.dynamicSmemBytes = (size_t)lmax * kNb * sizeof(double2) + 2 * (size_t)a.max_n * sizeof(int);
      cfg.stream = st;
      cudaLaunchAttribute attr[2];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = pc;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[1].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = chained ? 2 : 1;
      cudaError_t le = cudaLaunchKernelEx(&cfg, panel_cluster_kernel, a, jj, lmax);
      symhss::count_launches(1);
      return le;
    }
    if (smem_panel) {
      // the panel height shrinks with jj: fewer threads once the remaining rows allow it
      const int rows = a.max_n - jj;
      if (pthreads >= 1024 && rows > 512) panel_smem_kernel<1024, CT><<<a.njobs, 1024, panel_smem, st>>>(a, jj);
      else if (pthreads >= 512 && rows > 256) panel_smem_kernel<512, CT><<<a.njobs, 512, panel_smem, st>>>(a, jj);
      else panel_smem_kernel<256, CT><<<a.njobs, 256, panel_smem, st>>>(a, jj);
    } else {
      panel_kernel<CT><<<a.njobs, kPanelThreads, 0, st>>>(a, jj);
    }
    symhss::count_launches(1);
    return cudaGetLastError();
  };
  // lu_tc = 1: always; 2: launches of at least kTcMinJobs matrices (the lower tree levels, whose
  // many blocks fill the tensor-core product; at the top levels its per-launch latency and the
  // extra launches cost more than the FP64 updates they replace)
  const bool use_tc = (a.tc == 1 || (a.tc == 2 && a.njobs >= kTcMinJobs)) && a.zimg &&
                      a.zimg_bytes >= zgemm_lu_img_bytes(a.njobs, a.max_n);
  const int kOuter = (a.outer == 16 || a.outer == 32) ? a.outer : kOuterMax;
  const bool tc_path = sizeof(CT) == sizeof(double2) && use_tc && a.max_n > kOuter + kNb;
  // with rank-16 updates the chain is panel -> interchanges -> update -> panel, one stream
  const bool chain = tc_path && kOuter == kNb;
  if ((e = panel(0, s, chain)) != cudaSuccess) return e;
  if (tc_path) {
    // FP64: blocked by 64 columns (the order of a blocked right-looking LU).  Inside a block
    // the 16-column panels run as above with their interchanges applied to every column, but
    // their U-row solves and FP64 updates cover only the block's own columns.  At the block's
    // end its U rows for the columns right of it are solved (16 rows at a time), and
    // A22 -= L21 U12 (k = 64) runs on the tensor cores (zgemm_tc.cu).
    for (int j = 0; j < a.max_n; j += kNb) {
      const int J = (j / kOuter) * kOuter;
      const int rest = a.max_n - j - kNb;
      if (rest > 0) {
        // interchanges in every column; U rows only in the block's own columns (a block of
        // one panel: in every column right of it, so that no second pass is needed)
        e = narrow ? launch_chained(chain, swap_trsm_warp_kernel<CT, 8>, dim3(a.njobs, ncolblk8), dim3(128), 0, s, a,
                                    j, 0, chain ? a.max_n : J + kOuter, 1, 0)
                   : launch_chained(chain, swap_trsm_warp_kernel<CT, 32>, dim3(a.njobs, ncolblk), dim3(256), 0, s, a,
                                    j, 0, chain ? a.max_n : J + kOuter, 1, 0);
        symhss::count_launches(1);
        if (e != cudaSuccess) return e;
        const int pc = J + kOuter - (j + kNb);  // columns of the block right of this panel
        if (pc > 0) {
          update_kernel<CT><<<dim3(a.njobs, (rest + kTs - 1) / kTs, (pc + kTs - 1) / kTs), 256, 0, s>>>(a, j, 0, pc, -1);
          symhss::count_launches(1);
          if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
      }
      const int right = a.max_n - (J + kOuter);
      if (j + kNb == J + kOuter && right > 0) {
        // the block's U rows for the columns right of it, now that all its interchanges are
        // applied: 16-row solves, each followed by the update of the block rows below it
        const int rblk = (right + 31) / 32;  // blocks of 32 columns starting at J + kOuter
        for (int jj = J; kOuter > kNb && jj < J + kOuter; jj += kNb) {
          swap_trsm_warp_kernel<CT, 32><<<dim3(a.njobs, rblk), 256, 0, s>>>(a, jj, J + kOuter, a.max_n, 0, J + kOuter);
          symhss::count_launches(1);
          if ((e = cudaGetLastError()) != cudaSuccess) return e;
          const int r = J + kOuter - (jj + kNb);
          if (r > 0) {
            update_kernel<CT><<<dim3(a.njobs, (r + kTs - 1) / kTs, (right + kTs - 1) / kTs), 256, 0, s>>>(a, jj, r, -1, r);
            symhss::count_launches(1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
          }
        }
        ZgemmLaunch g;
        g.A = a.base; g.B = a.base; g.C = a.base;
        g.jobs = nullptr; g.tiles = nullptr;
        g.mode = ZGEMM_SUB;
        g.status = a.status;
        g.wait_ns = 0;
        g.derive = ZGEMM_LU_UPDATE;
        g.block_w = kOuter;
        g.inline_slice = kOuter <= 16;  // one 16-column chunk: sliced by the product's tiles
        g.chained = chain;
        g.lu_jobs = a.jobs;
        g.njobs = a.njobs;
        g.img = a.zimg;
        g.img_bytes = a.zimg_bytes;
        g.block_j = J;
        g.mtiles = (right + zgemm_tc_tile_rows() - 1) / zgemm_tc_tile_rows();
        g.ntiles_c = (right + zgemm_tc_tile_cols() - 1) / zgemm_tc_tile_cols();
        g.ntiles = a.njobs * g.mtiles * g.ntiles_c;
        if ((e = launch_zgemm_tc(g, s)) != cudaSuccess) return e;
      }
      if (j + kNb < a.max_n && (e = panel(j + kNb, s, chain)) != cudaSuccess) return e;
    }
    const int jlast = ((a.max_n - 1) / kNb) * kNb;
    e = narrow ? launch_chained(chain, swap_trsm_warp_kernel<CT, 8>, dim3(a.njobs, ncolblk8), dim3(128), 0, s, a,
                                jlast, 0, a.max_n, 1, 0)
               : launch_chained(chain, swap_trsm_warp_kernel<CT, 32>, dim3(a.njobs, ncolblk), dim3(256), 0, s, a,
                                jlast, 0, a.max_n, 1, 0);
    symhss::count_launches(1);
    return e;
  }
  for (int j = 0; j < a.max_n; j += kNb) {
    const int rest = a.max_n - j - kNb;
    if (rest <= 0) continue;
    swap_trsm_warp_kernel<CT, 32><<<dim3(a.njobs, ncolblk), 256, 0, s>>>(a, j, 0, a.max_n, 1, 0);
    symhss::count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int rtiles = (rest + kTs - 1) / kTs;
    const bool split = la != nullptr && rest > kTs;
    // first trailing tile column (all of it when not splitting)
    update_kernel<CT><<<dim3(a.njobs, rtiles, split ? 1 : rtiles), 256, 0, s>>>(a, j, 0, split ? kTs : -1, -1);
    symhss::count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!split) {
      if ((e = panel(j + kNb, s, false)) != cudaSuccess) return e;
      continue;
    }
    if ((e = cudaEventRecord(la->ready, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(la->side, la->ready, 0)) != cudaSuccess) return e;
    if ((e = panel(j + kNb, la->side, false)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(la->done, la->side)) != cudaSuccess) return e;
    const int ctiles = (rest - kTs + kTs - 1) / kTs;
    update_kernel<CT><<<dim3(a.njobs, rtiles, ctiles), 256, 0, s>>>(a, j, kTs, -1, -1);
    symhss::count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, la->done, 0)) != cudaSuccess) return e;
  }
  // the last panel's interchanges still have to reach the columns left of it
  const int jlast = ((a.max_n - 1) / kNb) * kNb;
  swap_trsm_warp_kernel<CT, 32><<<dim3(a.njobs, ncolblk), 256, 0, s>>>(a, jlast, 0, a.max_n, 1, 0);
  symhss::count_launches(1);
  return cudaGetLastError();
}

__global__ void pivot_reciprocal_kernel(const double2* a, int n, double2* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = cinv_pivot(a[i]);
}

cudaError_t launch_pivot_reciprocal(const double2* a, int n, double2* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  pivot_reciprocal_kernel<<<(n + 255) / 256, 256, 0, s>>>(a, n, out);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_getrf(const LuLaunch& a, cudaStream_t s) {
  return a.base32 ? getrf_impl<float2>(a, s) : getrf_impl<double2>(a, s);
}

}  // namespace symhss
