// Batched complex FP64 matrix product on the 5th-generation tensor cores (tcgen05), exact
// to FP64 rounding level: C = A B, C -= A B or C += A B with A m x k, B k x n, k <= 64, all
// complex128 and column-major.  Used by the blocked LU (trailing updates, triangular blocks
// applied through their inverses) and the multi-right-hand-side solves of the factorisation.
//
// Real form.  With A' = [Re A | Im A] (m x 2k) and, per complex column c of B, the two real
// columns [Re b_c; -Im b_c] and [Im b_c; Re b_c] (2k x 2), A' B' gives Re and Im of A b_c, so
// one real product with K' = 2k and N' = 2n computes the complex one.
//
// Exact slicing.  Every row i of A' is scaled by its largest binary exponent e_i and every
// column pair of B' by f_c; each entry x is then cut into eight signed 7-bit integers,
//   x = sign * sum_t d_t 2^(7 (7 - t)) 2^(e - 1078),   0 <= d_t <= 127,  t = 0..7,
// by integer operations on its FP64 bit pattern (only bits below 2^(e - 1078) are dropped).
// Each d_t is exact in bf16.  For the slice pairs (t, u) with t + u = s (s = 0..7; the pairs
// with s >= 8 weigh at most 2^-56 of the product and are dropped) the bf16 products d_t d'_u
// are summed over K' <= 128 into one FP32 accumulator G_s in tensor memory; every partial sum
// is an integer of magnitude below (s + 1) 128 127^2 <= 16516096 < 2^24, so the FP32
// accumulation is exact.  Then
//   (A B)_ic = sum_s G_s 2^(7 (7 - s)) 2^(e_i + f_c - 2107),
// recombined exactly in two int64 partial sums hi, lo (T = hi 2^28 + lo), rounded once to
// FP64 and scaled by a power of two: a few FP64 operations per real output instead of 4k FMAs.
//
// Kernels.  A launch is two kernels.  The slicing kernel cuts every 128-row block of A' and
// every 16-column block of B' once, in 16-column chunks of k, into the core-matrix order the
// MMA reads (eight slices per chunk, 64 KB for A', 16 KB for B'), in a scratch buffer the
// caller provides, together with the row and column exponents.  The product kernel then
// computes one 128 x 16 complex tile of C per thread block of 256 threads, two blocks per SM
// (256 tensor-memory columns, one 80 KB stage and 32K registers each), so that one block's
// epilogue overlaps the other's copies and MMAs.  One thread streams the tile's chunk images
// into the stage by bulk copies (cp.async.bulk, completing on an mbarrier) and issues the 36
// slice-pair products per K-step as 8 MMAs (M = 128, K = 16, N = 32 per B slice, the B slices
// j = 0 .. 7 - i of A slice i in one MMA; bf16 x bf16 -> FP32) into the eight groups of the
// accumulator.  The epilogue rounds T 2^(e_i + f_c - 2107) to FP64 by integer operations
// (one FP64 addition per real output for C -= AB and C += AB, none for C = AB).  Every wait is
// bounded by %globaltimer; after a timeout the block waits once more (bounded) for its copies
// and MMAs in flight, records ST_TIMEOUT, frees its tensor memory and exits.  A test hook
// (set_zgemm_timeout_probe) makes the last wait target a phase that no commit completes, so
// that this path can be exercised on purpose.
#include <stdint.h>

#include "common.cuh"

namespace symhss {

namespace {

constexpr int kMmaThreads = 256;  // product kernel (8 warps share the epilogue; two blocks per SM)
constexpr int kTileM = 128;       // rows of C per block
constexpr int kTileNc = 16;       // complex columns of C per block
constexpr int kNr = 2 * kTileNc;  // real columns of B' (MMA N)
constexpr int kSlices = 8;
constexpr int kGroups = 8;
constexpr int kChunkK = 16;                        // complex k per chunk (32 columns of A')
constexpr int kASliceBytes = kTileM * 32 * 2;      // 8192: one slice of the A' chunk
constexpr int kBSliceBytes = kNr * 32 * 2;         // 2048: one slice of the B' chunk
constexpr int kAChunkBytes = kSlices * kASliceBytes;               // 65536: A' chunk image
constexpr int kBChunkBytes = kSlices * kBSliceBytes;               // 16384: B' chunk image
constexpr int kStageBytes = kAChunkBytes + kBChunkBytes;           // 81920
constexpr int kMaxChunks = 4;                                      // k <= 64
constexpr int kTmemCols = kGroups * kNr;           // 256: two blocks per SM share the 512 columns
constexpr long long kWaitNs = 200ll * 1000 * 1000;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// no-swizzle K-major shared-memory matrix descriptor (core matrices of 8 rows x 16 bytes):
// LBO = byte distance of K-adjacent core matrices, SBO = of M/N-adjacent 8-row groups
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t make_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit_ns) {
  // non-blocking tests with a short back-off: the elapsed time is checked between tests, so
  // the limit holds however short it is (a blocking try may sleep until the phase completes)
  const unsigned long long t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
    if ((long long)(global_ns() - t0) > limit_ns) return false;
    __nanosleep(32);
  }
}

__device__ __forceinline__ int bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// the eight 7-bit slices of |x| relative to the biased exponent emax (>= that of x), each as an
// FP32 number whose upper half is its bf16 bit pattern, and the sign bit (0x8000) of x.  The
// fields come from two 32-bit halves of the aligned mantissa, and each 7-bit integer d becomes
// a float by one FP32 subtraction, (2^23 + d) - 2^23, exact (instead of an integer-to-float
// conversion per slice).
__device__ __forceinline__ void slice8(double x, int emax, uint32_t f[kSlices], uint32_t& sgn) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  uint64_t A = 0;
  if (E != 0 && emax != 0) {
    const uint64_t mant = ((uint64_t)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - emax + 3;  // A = |x| 2^(1078 - emax) < 2^56
    A = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
  }
  const uint32_t ahi = (uint32_t)(A >> 28), alo = (uint32_t)A & 0xFFFFFFFu;  // bits 55..28, 27..0
  sgn = bits < 0 ? 0x8000u : 0u;
#pragma unroll
  for (int t = 0; t < kSlices; ++t) {
    const uint32_t d = ((t < 4 ? ahi : alo) >> (21 - 7 * (t & 3))) & 0x7Fu;
    f[t] = __float_as_uint(__int_as_float(0x4B000000 | (int)d) - 8388608.0f);
  }
}

// an FP32 accumulator that holds an exact integer of magnitude below 2^22, as int: the
// integer lands in the low mantissa bits of v + 1.5 2^23
__device__ __forceinline__ int small_int(float v) { return __float_as_int(v + 12582912.0f) - 0x4B400000; }

// x 2^E for an integer-valued double x: exponent-field addition when x != 0 and the result
// is a normal number, else a multiplication by 2^E
__device__ __forceinline__ double scale2(double x, int E) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex != 0 && ex + E > 0 && ex + E < 2047) return __longlong_as_double(b + ((long long)E << 52));
  return (b & 0x7FFFFFFFFFFFFFFFll) == 0 ? x : ldexp(x, E);  // zero (tested on the bits) stays zero
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t v[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

// T 2^E rounded once to FP64 (to nearest, ties to even), for T = hi 2^28 + lo with |hi|,
// |lo| < 2^46.  T = h2 2^28 + l2 (0 <= l2 < 2^28) is cut to Ts = floor(T / 2^s) with s chosen
// so that Ts fits 64 bits (and, for s > 0, has at least 62 significant bits); the dropped bits
// of l2 become a sticky bit in the last place, which cannot move the rounding of a value of
// that length.  One correctly rounded integer-to-FP64 conversion then rounds T / 2^s, and the
// exponent field takes s + E.  (The conversion replaces about sixty integer instructions of an
// explicit cut and round, the larger part of the epilogue's issue time.)  A result outside the
// normal range (never for the products of this solver) is formed by FP64 operations instead.
// the FP64 path for results outside the normal range, as a call, so that its instructions are
// not if-converted into the common path (this GPU issues FP64 instructions slowly)
__device__ __noinline__ double recombine_slow(long long hi, long long lo, int E) {
  return scale2(fma((double)hi, 268435456.0, (double)lo), E);
}
__device__ __forceinline__ double recombine(long long hi, long long lo, int E) {
  const long long h2 = hi + (lo >> 28);
  const long long l2 = lo & 0xFFFFFFFll;
  const int mh = 63 - __clzll(h2 ^ (h2 >> 63));  // highest bit of |h2| (of |h2| - 1 if h2 < 0)
  const int s = mh > 34 ? mh - 34 : 0;           // |h2| 2^(28 - s) <= 2^63
  const long long Ts = ((long long)((unsigned long long)h2 << (28 - s)) + (l2 >> s)) |
                       ((l2 & ((1ll << s) - 1)) != 0 ? 1ll : 0ll);
  const long long db = __double_as_longlong(__ll2double_rn(Ts));
  const int be = (int)((db >> 52) & 0x7FF) + s + E;
  if (Ts == 0) return 0.0;
  if (be <= 0 || be >= 2047) return recombine_slow(hi, lo, E);
  return __longlong_as_double(db + ((long long)(s + E) << 52));
}

// the job of index jidx of a launch: explicit, or derived from the factorisation's job arrays
// (the block-J product of one matrix of the blocked LU or of the blocked triangular solves)
__device__ __forceinline__ ZgemmJob decode_job(const ZgemmLaunch& a, int jidx) {
  ZgemmJob jb;
  if (a.derive == ZGEMM_JOBS) return a.jobs[jidx];
  const int J = a.block_j;
  if (a.derive == ZGEMM_LU_UPDATE) {
    const LuJob lj = a.lu_jobs[jidx];
    const int W = a.block_w;
    jb.m = lj.n - J - W; jb.n = jb.m; jb.k = min(W, lj.n - J);
    jb.lda = jb.ldb = jb.ldc = lj.ld;
    jb.a_off = lj.a_off + (J + W) + (long long)J * lj.ld;
    jb.b_off = lj.a_off + J + (long long)(J + W) * lj.ld;
    jb.c_off = lj.a_off + (J + W) + (long long)(J + W) * lj.ld;
  } else if (a.derive == ZGEMM_RS_FWD_DIAG || a.derive == ZGEMM_RS_BWD_DIAG) {
    // the diagonal block's inverse (64 x 64, column-major, L's then U's per block) times the
    // block's rows of X, written over them (the slicing launch has read them first)
    const RsJob rj = a.rs_jobs[jidx];
    const int W = a.block_w;
    jb.m = jb.k = min(W, rj.n - J); jb.n = rj.nrhs;
    jb.lda = 64; jb.ldb = jb.ldc = rj.ldb;
    jb.a_off = (((long long)jidx * a.inv_nb + J / 64) * 2 + (a.derive == ZGEMM_RS_BWD_DIAG ? 1 : 0)) * 4096;
    jb.b_off = jb.c_off = rj.b_off + J;
  } else {
    const RsJob rj = a.rs_jobs[jidx];
    const int W = a.block_w;
    jb.k = min(W, rj.n - J); jb.n = rj.nrhs;
    jb.lda = rj.lda; jb.ldb = jb.ldc = rj.ldb;
    jb.b_off = rj.b_off + J;
    if (a.derive == ZGEMM_RS_FWD) {
      jb.m = rj.n - J - W;
      jb.a_off = rj.a_off + (J + W) + (long long)J * rj.lda;
      jb.c_off = rj.b_off + J + W;
    } else {
      jb.m = J;
      jb.a_off = rj.a_off + (long long)J * rj.lda;
      jb.c_off = rj.b_off;
    }
  }
  return jb;
}

// scratch layout: A' chunk images of every (job, row block), then B' chunk images of every
// (job, column block), then the row exponents (128 per row block), then the column exponents
// (32 per column block)
struct ImgLayout {
  unsigned char* a;
  unsigned char* b;
  int* ea;
  int* fb;
};
__host__ __device__ __forceinline__ ImgLayout img_layout(unsigned char* img, int njobs, int mtiles, int ntiles) {
  ImgLayout L;
  L.a = img;
  L.b = L.a + (size_t)njobs * mtiles * kMaxChunks * kAChunkBytes;
  L.ea = reinterpret_cast<int*>(L.b + (size_t)njobs * ntiles * kMaxChunks * kBChunkBytes);
  L.fb = L.ea + (size_t)njobs * mtiles * kTileM;
  return L;
}

// the eight slices of eight values (relative to biased exponent emax) packed as bf16 pairs:
// one byte permutation joins slice t of two neighbouring values.  A zero slice of a negative
// value is -0, whose products add nothing to the sums.
__device__ __forceinline__ void slice_pack8(const double x[8], int emax, uint32_t pk[kSlices][4]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    uint32_t fa[kSlices], fb[kSlices], sa, sb;
    slice8(x[2 * m], emax, fa, sa);
    slice8(x[2 * m + 1], emax, fb, sb);
    const uint32_t sg = sa | (sb << 16);
#pragma unroll
    for (int t = 0; t < kSlices; ++t) pk[t][m] = __byte_perm(fa[t], fb[t], 0x7632) | sg;
  }
}

// Slicing kernel (512 threads): blocks [0, njobs mtiles) cut row blocks of A', the rest column
// blocks of B'.  Every thread loads its share of the block once (all loads in flight together),
// takes the exponents from registers and writes its slices.
constexpr int kSliceThreads = 512;

__global__ void __launch_bounds__(kSliceThreads) zslice_kernel(const ZgemmLaunch a) {
  pdl_enter();
  __shared__ int s_e[kMaxChunks][kTileM];
  const ImgLayout L = img_layout(a.img, a.njobs, a.mtiles, a.ntiles_c);
  const int nA = a.njobs * a.mtiles;
  const int tid = threadIdx.x;
  if ((int)blockIdx.x < nA) {
    const int jidx = blockIdx.x / a.mtiles, mt = blockIdx.x - jidx * a.mtiles;
    const ZgemmJob jb = decode_job(a, jidx);
    const int r0 = mt * kTileM;
    if (jb.m <= 0 || jb.n <= 0 || jb.k <= 0 || r0 >= jb.m) return;  // uniform per block
    const int m = jb.m, K = jb.k;
    const double2* A = a.A + jb.a_off;
    // thread (rt, ch): row r0 + rt, the 16 values of k chunk ch
    const int rt = tid & (kTileM - 1), ch = tid >> 7;
    const int row = r0 + rt;
    double2 v[kChunkK];
    int e = 0;
#pragma unroll
    for (int q = 0; q < kChunkK; ++q) {
      const int k = ch * kChunkK + q;
      v[q] = (row < m && k < K) ? A[row + (long long)k * jb.lda] : make_double2(0.0, 0.0);
      e = max(e, max(bexp(v[q].x), bexp(v[q].y)));
    }
    s_e[ch][rt] = e;
    __syncthreads();
    const int ea = max(max(s_e[0][rt], s_e[1][rt]), max(s_e[2][rt], s_e[3][rt]));  // the row's largest
    const size_t blk = (size_t)jidx * a.mtiles + mt;
    if (ch == 0) L.ea[blk * kTileM + rt] = ea;
    if (ch * kChunkK >= K) return;  // no such chunk
    unsigned char* img = L.a + (blk * kMaxChunks + ch) * kAChunkBytes;
    // core rows q = 0, 1 hold Re a(row, k0 + 8q + e), q = 2, 3 hold Im of the same k
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int h = q & 1, part = q >> 1;
      double x[8];
#pragma unroll
      for (int e8 = 0; e8 < 8; ++e8) x[e8] = part ? v[8 * h + e8].y : v[8 * h + e8].x;
      uint32_t pk[kSlices][4];
      slice_pack8(x, ea, pk);
#pragma unroll
      for (int t = 0; t < kSlices; ++t)
        *reinterpret_cast<uint4*>(img + t * kASliceBytes + (rt >> 3) * 512 + q * 128 + (rt & 7) * 16) =
            make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
    }
    return;
  }
  const int bidx = blockIdx.x - nA;
  const int jidx = bidx / a.ntiles_c, nt = bidx - jidx * a.ntiles_c;
  const ZgemmJob jb = decode_job(a, jidx);
  const int c0 = nt * kTileNc;
  if (jb.m <= 0 || jb.n <= 0 || jb.k <= 0 || c0 >= jb.n) return;  // uniform per block
  const int n = jb.n, K = jb.k;
  const double2* B = a.B + jb.b_off;
  // thread (c, ch, comp, kh): component comp (Re / Im) of b(16 ch + 8 kh .. + 7, c0 + c); the
  // 16 threads of a column are 16 consecutive lanes (whole warps beyond the block's columns)
  const int c = tid >> 4, ch = (tid >> 2) & 3, comp = (tid >> 1) & 1, kh = tid & 1;
  if (c >= kTileNc) return;
  const int col = c0 + c;
  double x[8];
  int fb = 0;
#pragma unroll
  for (int e8 = 0; e8 < 8; ++e8) {
    const int k = ch * kChunkK + 8 * kh + e8;
    const double2 v = (col < n && k < K) ? B[k + (long long)col * jb.ldb] : make_double2(0.0, 0.0);
    x[e8] = comp ? v.y : v.x;
    fb = max(fb, bexp(x[e8]));
  }
#pragma unroll
  for (int o = 1; o < 16; o <<= 1) fb = max(fb, __shfl_xor_sync(0xffffffffu, fb, o));  // the column's largest
  const size_t blk = (size_t)jidx * a.ntiles_c + nt;
  if ((tid & 15) == 0) L.fb[blk * kTileNc + c] = fb;
  if (ch * kChunkK >= K) return;  // no such chunk
  unsigned char* img = L.b + (blk * kMaxChunks + ch) * kBChunkBytes;
  // B' columns of complex column c: n' = 2c holds [Re b; -Im b], n' = 2c + 1 holds [Im b; Re b]
  // (core rows q = 0, 1: the k halves paired with Re a; q = 2, 3: with Im a).  Re b goes to
  // (2c, kh) and (2c + 1, kh + 2); Im b to (2c + 1, kh) and, sign bits flipped, (2c, kh + 2)
  const int np1 = 2 * c + comp, q1 = kh;
  const int np2 = 2 * c + 1 - comp, q2 = kh + 2;
  const uint32_t flip2 = comp ? 0x80008000u : 0u;
  uint32_t pk[kSlices][4];
  slice_pack8(x, fb, pk);
#pragma unroll
  for (int t = 0; t < kSlices; ++t) {
    unsigned char* sl = img + t * kBSliceBytes;
    *reinterpret_cast<uint4*>(sl + (np1 >> 3) * 512 + q1 * 128 + (np1 & 7) * 16) =
        make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
    // a flipped zero slice is -0: its products add nothing to the sums
    *reinterpret_cast<uint4*>(sl + (np2 >> 3) * 512 + q2 * 128 + (np2 & 7) * 16) =
        make_uint4(pk[t][0] ^ flip2, pk[t][1] ^ flip2, pk[t][2] ^ flip2, pk[t][3] ^ flip2);
  }
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

__global__ void __launch_bounds__(kMmaThreads, 2) zgemm_tc_kernel(const ZgemmLaunch a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  pdl_enter();
  __shared__ __align__(8) uint64_t bar_mma[2];
  __shared__ __align__(8) uint64_t bar_load[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_fail, s_last;
  __shared__ int s_fexp[kTileNc];
  __shared__ int s_e[kTileM];
  int jidx, mt, nt;
  if (a.derive == ZGEMM_JOBS) {
    const ZgemmTile tl = a.tiles[blockIdx.x];
    jidx = tl.job;
    mt = tl.mt;
    nt = tl.nt;
  } else {
    const int per = a.mtiles * a.ntiles_c;
    jidx = blockIdx.x / per;
    const int rem = blockIdx.x - jidx * per;
    mt = rem / a.ntiles_c;
    nt = rem - mt * a.ntiles_c;
  }
  const ZgemmJob jb = decode_job(a, jidx);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = mt * kTileM, c0 = nt * kTileNc;
  // idle tile (a derived job smaller than the launch's largest, or a tile outside the
  // image blocks): leave before any barrier
  if (jb.m <= 0 || jb.n <= 0 || jb.k <= 0 || r0 >= jb.m || c0 >= jb.n || mt >= a.mtiles || nt >= a.ntiles_c ||
      jidx >= a.njobs)
    return;
  const int m = jb.m, n = jb.n, K = jb.k;
  double2* C = a.C + jb.c_off;
  const ImgLayout L = img_layout(a.img, a.njobs, a.mtiles, a.ntiles_c);
  const size_t ablk = (size_t)jidx * a.mtiles + mt, bblk = (size_t)jidx * a.ntiles_c + nt;
  const unsigned char* gA = L.a + ablk * kMaxChunks * kAChunkBytes;
  const unsigned char* gB = L.b + bblk * kMaxChunks * kBChunkBytes;
  if (!a.inline_slice) {
    if (tid < kTileM) s_e[tid] = L.ea[ablk * kTileM + tid];
    if (tid < kTileNc) s_fexp[tid] = L.fb[bblk * kTileNc + tid];
  }
  // inline slicing: the operand loads are issued before the setup below, which their latency
  // then overlaps.  A: thread (rt, half) holds a(r0 + rt, 8 half .. + 7); B: thread (bc, comp,
  // kh), tid < 64, component comp of b(8 kh .. + 7, c0 + bc)
  double re[8], im[8], xb[8];
  const int rt = tid & (kTileM - 1), half = tid >> 7;
  const int bc = tid >> 2, comp = (tid >> 1) & 1, kh = tid & 1;
  if (a.inline_slice) {
    const double2* A = a.A + jb.a_off;
    const int row = r0 + rt;
#pragma unroll
    for (int e8 = 0; e8 < 8; ++e8) {
      const int k = 8 * half + e8;
      const double2 v = (row < m && k < K) ? A[row + (long long)k * jb.lda] : make_double2(0.0, 0.0);
      re[e8] = v.x;
      im[e8] = v.y;
    }
    if (tid < 4 * kTileNc) {
      const double2* B = a.B + jb.b_off;
#pragma unroll
      for (int e8 = 0; e8 < 8; ++e8) {
        const int k = 8 * kh + e8;
        const double2 v = (c0 + bc < n && k < K) ? B[k + (long long)(c0 + bc) * jb.ldb] : make_double2(0.0, 0.0);
        xb[e8] = comp ? v.y : v.x;
      }
    }
  }
  if (a.mode != ZGEMM_SET && warp == 1) {
    // the old values of the tile's columns into L2 while the MMAs run (one column per lane)
    const int col = c0 + lane, rows = min(kTileM, m - r0);
    if (lane < kTileNc && col < n && rows > 0)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                   :: "l"(C + r0 + (long long)col * jb.ldc), "r"((uint32_t)(rows * sizeof(double2))) : "memory");
  }
  if (tid == 0) {
    s_fail = 0;
    s_last = -1;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_mma[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_load[i])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base_s)), "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_s;
  const int nch = (K + kChunkK - 1) / kChunkK;

  if (a.inline_slice) {
    // one chunk (k <= 16): the block slices its own operands into the stage (row / column
    // exponents over this chunk, which is all of k), no images and no slicing launch
    __shared__ int s_eh[2][kTileM];
    int e = 0;
#pragma unroll
    for (int e8 = 0; e8 < 8; ++e8) e = max(e, max(bexp(re[e8]), bexp(im[e8])));
    s_eh[half][rt] = e;
    int fb = 0;
    if (tid < 4 * kTileNc) {
#pragma unroll
      for (int e8 = 0; e8 < 8; ++e8) fb = max(fb, bexp(xb[e8]));
    }
    if (warp < 2) {  // the column's largest over its four threads (lanes 4c .. 4c + 3)
      fb = max(fb, __shfl_xor_sync(0xffffffffu, fb, 1));
      fb = max(fb, __shfl_xor_sync(0xffffffffu, fb, 2));
      if (tid < 4 * kTileNc && (tid & 3) == 0) s_fexp[bc] = fb;
    }
    __syncthreads();
    const int ea = max(s_eh[0][rt], s_eh[1][rt]);
    if (half == 0) s_e[rt] = ea;
    unsigned char* sA = smem;
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      uint32_t pk[kSlices][4];
      slice_pack8(part ? im : re, ea, pk);
      const int q = half + 2 * part;
#pragma unroll
      for (int t = 0; t < kSlices; ++t)
        *reinterpret_cast<uint4*>(sA + t * kASliceBytes + (rt >> 3) * 512 + q * 128 + (rt & 7) * 16) =
            make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
    }
    if (tid < 4 * kTileNc) {
      unsigned char* sB = smem + kAChunkBytes;
      const int np1 = 2 * bc + comp, q1 = kh, np2 = 2 * bc + 1 - comp, q2 = kh + 2;
      const uint32_t flip2 = comp ? 0x80008000u : 0u;
      uint32_t pk[kSlices][4];
      slice_pack8(xb, s_fexp[bc], pk);
#pragma unroll
      for (int t = 0; t < kSlices; ++t) {
        unsigned char* sl = sB + t * kBSliceBytes;
        *reinterpret_cast<uint4*>(sl + (np1 >> 3) * 512 + q1 * 128 + (np1 & 7) * 16) =
            make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
        *reinterpret_cast<uint4*>(sl + (np2 >> 3) * 512 + q2 * 128 + (np2 & 7) * 16) =
            make_uint4(pk[t][0] ^ flip2, pk[t][1] ^ flip2, pk[t][2] ^ flip2, pk[t][3] ^ flip2);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sa = smem_u32(smem), sb = sa + kAChunkBytes;
      const uint64_t ad0 = make_desc(sa, 128, 512), bd0 = make_desc(sb, 128, 512);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
        for (int i = 0; i < kSlices; ++i) {
          const uint64_t ad = ad0 + (uint64_t)((i * kASliceBytes + kk * 256) >> 4);
          const uint64_t bd = bd0 + (uint64_t)((kk * 256) >> 4);
          const uint32_t acc = (kk > 0 || i > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
              :: "r"(tmem + (uint32_t)(i * kNr)), "l"(ad), "l"(bd), "r"(make_idesc(kTileM, kNr * (kSlices - i))),
                 "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&bar_mma[0])) : "memory");
      s_last = 0;
    }
  } else if (tid == 0) {
    // one thread streams the chunk images and issues the MMAs: chunk c lives in stage c % 2;
    // the copy of chunk c + 1 (c >= 1) is issued once the MMAs of chunk c - 1 have released
    // its stage, so that it overlaps the MMAs of chunk c
    const uint32_t sbase = smem_u32(smem);
    int issued = 0, waited = 0, fail = 0;
    auto issue = [&](int ch) {
      const uint32_t bar = smem_u32(&bar_load[0]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(kStageBytes) : "memory");
      bulk_load(sbase, gA + (size_t)ch * kAChunkBytes, kAChunkBytes, bar);
      bulk_load(sbase + kAChunkBytes, gB + (size_t)ch * kBChunkBytes, kBChunkBytes, bar);
      issued = ch + 1;
    };
    issue(0);
    for (int ch = 0; ch < nch; ++ch) {
      if (!mbar_wait(smem_u32(&bar_load[0]), (uint32_t)(ch & 1), a.wait_ns)) { fail = 1; break; }
      waited = ch + 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sA = sbase, sB = sA + kAChunkBytes;
      // descriptors differ only in their address field (address / 16 < 2^14 in shared memory)
      const uint64_t ad0 = make_desc(sA, 128, 512), bd0 = make_desc(sB, 128, 512);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        // A slice i times B slices 0 .. 7 - i in one MMA of N = 32 (8 - i): the B slices lie
        // next to each other along N (same 512-byte stride between 8-row groups), and so do the
        // accumulator groups i .. 7 in tensor memory; slice pairs with i + j >= 8 are never formed
#pragma unroll
        for (int i = 0; i < kSlices; ++i) {
          const int nb = kSlices - i;
          const uint64_t ad = ad0 + (uint64_t)((i * kASliceBytes + kk * 256) >> 4);
          const uint64_t bd = bd0 + (uint64_t)((kk * 256) >> 4);
          const uint32_t acc = (ch > 0 || kk > 0 || i > 0) ? 1u : 0u;  // i = 0 opens every group
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
              :: "r"(tmem + (uint32_t)(i * kNr)), "l"(ad), "l"(bd), "r"(make_idesc(kTileM, kNr * nb)), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&bar_mma[0])) : "memory");
      s_last = ch;
      if (ch + 1 < nch) {
        // one stage: the MMAs of chunk ch release it for chunk ch + 1 (the other block on this
        // SM keeps the tensor pipe busy meanwhile)
        if (!mbar_wait(smem_u32(&bar_mma[0]), (uint32_t)(ch & 1), a.wait_ns)) {
          fail = 1;
          break;
        }
        issue(ch + 1);
      }
    }
    if (fail) {
      // drain: every copy still in flight (bounded), before the stages are given up
      for (int c = waited; c < issued; ++c) mbar_wait(smem_u32(&bar_load[0]), (uint32_t)(c & 1), kWaitNs);
      s_fail = 1;
    }
  }
  __syncthreads();
  // wait for the last committed chunk (its commit covers every earlier MMA of the block)
  if (tid == 0 && s_last >= 0) {
    const int lc = s_last;
    const uint32_t bar = smem_u32(&bar_mma[0]);
    const uint32_t par = (uint32_t)(lc & 1);
    if (s_fail) {
      mbar_wait(bar, par, kWaitNs);  // drain the MMAs still in flight
    } else if (a.probe_timeout) {
      // test hook: after the real phase, wait for the next one, which nothing completes
      mbar_wait(bar, par, kWaitNs);
      if (!mbar_wait(bar, par ^ 1u, a.wait_ns)) s_fail = 1;
    } else if (!mbar_wait(bar, par, a.wait_ns)) {
      s_fail = 1;
      mbar_wait(bar, par, kWaitNs);  // drain
    }
  }
  if (tid == 0 && s_fail) atomicOr(a.status, ST_TIMEOUT);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");

  if (!s_fail) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows r0 + 32 (w % 4) + lane) and
    // the complex columns 8 (w / 4) .. + 7 of the tile
    const int er = r0 + 32 * (warp & 3) + lane;
    const int eea = s_e[er - r0];
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
    for (int cq = 0; cq < 2; ++cq) {
      const int cb = 2 * (warp >> 2) + cq;  // 4 complex (8 real) columns
      if (c0 + cb * 4 >= n) break;           // uniform per warp
      // the old values first, so that their loads overlap the tensor-memory reads
      double2 old4[4];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int col = c0 + cb * 4 + cc;
        old4[cc] = (a.mode != ZGEMM_SET && er < m && col < n) ? C[er + (long long)col * jb.ldc] : make_double2(0.0, 0.0);
      }
      uint32_t v[kGroups][8];
#pragma unroll
      for (int s = 0; s < kGroups; ++s) tmem_ld8(lane_base + (uint32_t)(s * kNr + cb * 8), v[s]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      // the group sums as integers: one FP32 addition each when all are below 2^22 (the
      // common case), else the conversion instruction
      bool small = true;
#pragma unroll
      for (int s = 0; s < kGroups; ++s)
#pragma unroll
        for (int q = 0; q < 8; ++q) small = small && fabsf(__uint_as_float(v[s][q])) < 4194304.0f;
      int gi[kGroups][8];
      if (small) {
#pragma unroll
        for (int s = 0; s < kGroups; ++s)
#pragma unroll
          for (int q = 0; q < 8; ++q) gi[s][q] = small_int(__uint_as_float(v[s][q]));
      } else {
#pragma unroll
        for (int s = 0; s < kGroups; ++s)
#pragma unroll
          for (int q = 0; q < 8; ++q) gi[s][q] = __float2int_rn(__uint_as_float(v[s][q]));
      }
      if (er < m) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int c = cb * 4 + cc, col = c0 + c;
          if (col >= n) continue;
          const int fb = s_fexp[c];
          // times 2^(e_i + f_c - 2107), folded into the rounding
          const int E = eea + fb - 2107;
          double pr[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int q = 2 * cc + h;
            // below 2^22 the pairs g0 2^7 + g1 fit 32 bits
            const long long hi = small ? (long long)(gi[0][q] * 128 + gi[1][q]) * 16384 + (gi[2][q] * 128 + gi[3][q])
                                       : ((((long long)gi[0][q] * 128 + gi[1][q]) * 128 + gi[2][q]) * 128) + gi[3][q];
            const long long lo = small ? (long long)(gi[4][q] * 128 + gi[5][q]) * 16384 + (gi[6][q] * 128 + gi[7][q])
                                       : ((((long long)gi[4][q] * 128 + gi[5][q]) * 128 + gi[6][q]) * 128) + gi[7][q];
            const double rv = recombine(hi, lo, E);
            pr[h] = (eea == 0 || fb == 0) ? 0.0 : rv;
          }
          const double2 o = old4[cc];
          double2* cp = C + er + (long long)col * jb.ldc;
          if (a.mode == ZGEMM_SET) *cp = make_double2(pr[0], pr[1]);  // the mode is uniform over the launch
          else if (a.mode == ZGEMM_SUB) *cp = make_double2(o.x - pr[0], o.y - pr[1]);
          else *cp = make_double2(o.x + pr[0], o.y + pr[1]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
}

long long g_zgemm_wait_ns = kWaitNs;
int g_zgemm_probe = 0;

}  // namespace

void set_zgemm_wait_ns(long long ns) { g_zgemm_wait_ns = ns > 0 ? ns : kWaitNs; }
void set_zgemm_timeout_probe(int on) { g_zgemm_probe = on ? 1 : 0; }

int zgemm_tc_tile_rows() { return kTileM; }
int zgemm_tc_tile_cols() { return kTileNc; }
int zgemm_tc_max_k() { return kMaxChunks * kChunkK; }

long long zgemm_img_bytes(int njobs, int mtiles, int ntiles) {
  if (njobs <= 0 || mtiles <= 0 || ntiles <= 0) return 0;
  return (long long)njobs * ((long long)mtiles * (kMaxChunks * (long long)kAChunkBytes + kTileM * 4) +
                             (long long)ntiles * (kMaxChunks * (long long)kBChunkBytes + kTileNc * 4));
}

long long zgemm_img_bytes_for(int njobs, int max_m, int max_n) {
  if (max_m <= 0 || max_n <= 0) return 0;
  return zgemm_img_bytes(njobs, (max_m + kTileM - 1) / kTileM, (max_n + kTileNc - 1) / kTileNc);
}

long long zgemm_lu_img_bytes(int njobs, int max_n) { return zgemm_img_bytes_for(njobs, max_n - 16, max_n - 16); }
long long zgemm_rs_img_bytes(int njobs, int max_n, int max_rhs) { return zgemm_img_bytes_for(njobs, max_n, max_rhs); }

cudaError_t launch_zgemm_tc(const ZgemmLaunch& a_in, cudaStream_t s) {
  if (a_in.ntiles <= 0) return cudaSuccess;
  ZgemmLaunch a = a_in;
  if (a.njobs <= 0 || a.mtiles <= 0 || a.ntiles_c <= 0) return cudaErrorInvalidValue;
  // tiles slice their own operands only where every k is one chunk: the LU update of a
  // block of at most 16 columns (the kernel takes chunk 0 alone on that path)
  if (a.inline_slice && !(a.derive == ZGEMM_LU_UPDATE && a.block_w > 0 && a.block_w <= kChunkK))
    return cudaErrorInvalidValue;
  if (!a.inline_slice && (!a.img || a.img_bytes < zgemm_img_bytes(a.njobs, a.mtiles, a.ntiles_c) ||
                          (reinterpret_cast<uintptr_t>(a.img) & 15)))
    return cudaErrorInvalidValue;
  a.wait_ns = g_zgemm_wait_ns;
  a.probe_timeout = g_zgemm_probe;
  cudaError_t e;
  if (!a.inline_slice) {
    e = launch_chained(a.chained, zslice_kernel, dim3(a.njobs * (a.mtiles + a.ntiles_c)), dim3(kSliceThreads), 0, s,
                       a);
    symhss::count_launches(1);
    if (e != cudaSuccess) return e;
  }
  const int smem = kStageBytes;
  e = cudaFuncSetAttribute(zgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  // after the slicing kernel: always its programmatic dependent
  e = launch_chained(a.chained || !a.inline_slice, zgemm_tc_kernel, dim3(a.ntiles), dim3(kMmaThreads), smem, s, a);
  symhss::count_launches(1);
  return e;
}

}  // namespace symhss
