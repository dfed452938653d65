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
// Kernel.  One thread block of 256 threads computes a 128 x 32 complex tile of C.  For each
// chunk of 16 complex columns of A (32 columns of A'), two threads per row slice the row's
// halves of the chunk and every thread one core row of the tile's B chunk into shared memory
// (two stages, 96 KB each, in the core-matrix order the MMA reads); one thread issues the
// 36 slice-pair MMAs per K-step
// (M = 128, N = 64, K = 16, bf16 x bf16 -> FP32) into the eight groups of a 512-column
// tensor-memory accumulator and commits them to the stage's mbarrier; slicing of the next
// chunk overlaps those MMAs.  Every wait is bounded by %globaltimer; after a timeout the block
// waits once more (bounded) for its MMAs in flight, records ST_TIMEOUT, frees its tensor
// memory and exits.  A test hook (set_zgemm_timeout_probe) makes the last wait target a
// phase that no commit completes, so that this path can be exercised on purpose.
#include <stdint.h>

#include "common.cuh"

namespace symhss {

namespace {

constexpr int kThreads = 256;
constexpr int kTileM = 128;       // rows of C per block
constexpr int kTileNc = 32;       // complex columns of C per block
constexpr int kNr = 2 * kTileNc;  // real columns of B' (MMA N)
constexpr int kSlices = 8;
constexpr int kGroups = 8;
constexpr int kChunkK = 16;                        // complex k per chunk (32 columns of A')
constexpr int kASliceBytes = kTileM * 32 * 2;      // 8192: one slice of the A' chunk
constexpr int kBSliceBytes = kNr * 32 * 2;         // 4096: one slice of the B' chunk
constexpr int kStageBytes = kSlices * (kASliceBytes + kBSliceBytes);  // 98304
constexpr int kTmemCols = kGroups * kNr;           // 512
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

// the eight 7-bit slices of x relative to the biased exponent emax (>= that of x), as bf16
// bit patterns with the sign of x.  The fields come from two 32-bit halves of the aligned
// mantissa, and each 7-bit integer d becomes a float by one FP32 subtraction,
// (2^23 + d) - 2^23, exact (instead of an integer-to-float conversion per slice).
__device__ __forceinline__ void slice8(double x, int emax, uint32_t out[kSlices], bool negate = false) {
  // the sign is taken from the bit pattern (negation flips it: no FP64 instruction)
  const long long bits = __double_as_longlong(x) ^ (negate ? (long long)0x8000000000000000ull : 0ll);
  const int E = (int)((bits >> 52) & 0x7FF);
  uint64_t A = 0;
  if (E != 0 && emax != 0) {
    const uint64_t mant = ((uint64_t)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - emax + 3;  // A = |x| 2^(1078 - emax) < 2^56
    A = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
  }
  const uint32_t ahi = (uint32_t)(A >> 28), alo = (uint32_t)A & 0xFFFFFFFu;  // bits 55..28, 27..0
  const uint32_t sgn = bits < 0 ? 0x8000u : 0u;
#pragma unroll
  for (int t = 0; t < kSlices; ++t) {
    const uint32_t d = ((t < 4 ? ahi : alo) >> (21 - 7 * (t & 3))) & 0x7Fu;
    const float f = __int_as_float(0x4B000000 | (int)d) - 8388608.0f;
    out[t] = d ? ((__float_as_uint(f) >> 16) | sgn) : 0u;
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

__global__ void __launch_bounds__(kThreads, 1) zgemm_tc_kernel(const ZgemmLaunch a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_mma[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_fail, s_last;
  __shared__ int s_fexp[kTileNc];
  __shared__ int s_eh[2][kTileM];
  ZgemmJob jb;
  int mt, nt;
  if (a.derive == ZGEMM_JOBS) {
    const ZgemmTile tl = a.tiles[blockIdx.x];
    jb = a.jobs[tl.job];
    mt = tl.mt;
    nt = tl.nt;
  } else {
    // the block-J product of one factorisation job (64-column blocks of the blocked LU and
    // of the blocked triangular solves)
    const int per = a.mtiles * a.ntiles_c;
    const int jidx = blockIdx.x / per, rem = blockIdx.x - jidx * per;
    mt = rem / a.ntiles_c;
    nt = rem - mt * a.ntiles_c;
    const int J = a.block_j;
    if (a.derive == ZGEMM_LU_UPDATE) {
      const LuJob lj = a.lu_jobs[jidx];
      jb.m = lj.n - J - 64; jb.n = jb.m; jb.k = min(64, lj.n - J);
      jb.lda = jb.ldb = jb.ldc = lj.ld;
      jb.a_off = lj.a_off + (J + 64) + (long long)J * lj.ld;
      jb.b_off = lj.a_off + J + (long long)(J + 64) * lj.ld;
      jb.c_off = lj.a_off + (J + 64) + (long long)(J + 64) * lj.ld;
    } else {
      const RsJob rj = a.rs_jobs[jidx];
      jb.k = min(64, rj.n - J); jb.n = rj.nrhs;
      jb.lda = rj.lda; jb.ldb = jb.ldc = rj.ldb;
      jb.b_off = rj.b_off + J;
      if (a.derive == ZGEMM_RS_FWD) {
        jb.m = rj.n - J - 64;
        jb.a_off = rj.a_off + (J + 64) + (long long)J * rj.lda;
        jb.c_off = rj.b_off + J + 64;
      } else {
        jb.m = J;
        jb.a_off = rj.a_off + (long long)J * rj.lda;
        jb.c_off = rj.b_off;
      }
    }
  }
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = mt * kTileM, c0 = nt * kTileNc;
  // idle tile of a derived job (smaller than the launch's largest): leave before any barrier
  if (jb.m <= 0 || jb.n <= 0 || jb.k <= 0 || r0 >= jb.m || c0 >= jb.n) return;
  const int m = jb.m, n = jb.n, K = jb.k;
  const double2* A = a.A + jb.a_off;
  const double2* B = a.B + jb.b_off;
  double2* C = a.C + jb.c_off;
  // slicing roles: thread (rt, half) slices row r0 + rt of A, k-half `half` of every chunk
  const int rt = tid & (kTileM - 1), half = tid >> 7;
  const int row = r0 + rt;

  // exponents: rows of A (two threads per row, halves of k), columns of B (8 threads each);
  // the loads of a thread are independent and unrolled so that many are in flight
  {
    int e = 0;
    if (row < m) {
#pragma unroll 8
      for (int k = half; k < K; k += 2) {
        const double2 v = A[row + (long long)k * jb.lda];
        e = max(e, max(bexp(v.x), bexp(v.y)));
      }
    }
    s_eh[half][rt] = e;
    const int c = tid >> 3, q = tid & 7;
    int fb = 0;
    if (c0 + c < n) {
#pragma unroll 8
      for (int k = q; k < K; k += 8) {
        const double2 v = B[k + (long long)(c0 + c) * jb.ldb];
        fb = max(fb, max(bexp(v.x), bexp(v.y)));
      }
    }
    fb = max(fb, __shfl_xor_sync(0xffffffffu, fb, 1));
    fb = max(fb, __shfl_xor_sync(0xffffffffu, fb, 2));
    fb = max(fb, __shfl_xor_sync(0xffffffffu, fb, 4));
    if (q == 0) s_fexp[c] = fb;
  }
  if (tid == 0) {
    s_fail = 0;
    s_last = -1;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_mma[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_mma[1])));
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
  const int ea = max(s_eh[0][rt], s_eh[1][rt]);  // this row's largest biased exponent
  const uint32_t idesc = make_idesc(kTileM, kNr);
  const int nch = (K + kChunkK - 1) / kChunkK;

  for (int ch = 0; ch < nch; ++ch) {
    const int st = ch & 1;
    unsigned char* sA = smem + st * kStageBytes;
    unsigned char* sB = sA + kSlices * kASliceBytes;
    if (ch >= 2) {  // the MMAs of chunk ch - 2 read this stage: wait for them
      if (tid == 0 && !mbar_wait(smem_u32(&bar_mma[st]), (uint32_t)(((ch - 2) >> 1) & 1), a.wait_ns)) s_fail = 1;
      __syncthreads();
      if (s_fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
    const int k0 = ch * kChunkK;
    // A' chunk: core rows q = 0, 1 hold Re a(row, k0 + 8q + e), q = 2, 3 hold Im of the same
    // k; thread (rt, half) writes the rows q = half and q = half + 2 of its row
    {
      const int h = half;
      double re[8], im[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + 8 * h + e;
        double2 v = make_double2(0.0, 0.0);
        if (row < m && k < K) v = A[row + (long long)k * jb.lda];
        re[e] = v.x;
        im[e] = v.y;
      }
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        uint32_t pk[kSlices][4];
#pragma unroll
        for (int t = 0; t < kSlices; ++t) pk[t][0] = pk[t][1] = pk[t][2] = pk[t][3] = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          uint32_t sl[kSlices];
          slice8(part ? im[e] : re[e], ea, sl);
#pragma unroll
          for (int t = 0; t < kSlices; ++t) pk[t][e >> 1] |= sl[t] << (16 * (e & 1));
        }
        const int q = h + 2 * part;
#pragma unroll
        for (int t = 0; t < kSlices; ++t)
          *reinterpret_cast<uint4*>(sA + t * kASliceBytes + (rt >> 3) * 512 + q * 128 + (rt & 7) * 16) =
              make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
      }
    }
    // B' chunk: thread -> real column n' = tid / 4 (complex column c = n' / 2, part = n' % 2)
    // and core row q = tid % 4 (k half kh = q % 2; q < 2: rows paired with Re a, else Im a)
    {
      const int np = tid >> 2, q = tid & 3;
      const int c = np >> 1, part = np & 1, kh = q & 1, wim = q >> 1;
      const int col = c0 + c;
      const int fb = s_fexp[c];
      double x[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + 8 * kh + e;
        double2 v = make_double2(0.0, 0.0);
        if (col < n && k < K) v = B[k + (long long)col * jb.ldb];
        // rows with Re a: (Re b | Im b); rows with Im a: (-Im b | Re b), the sign applied below
        x[e] = wim ? (part ? v.x : v.y) : (part ? v.y : v.x);
      }
      const bool neg = wim && !part;
      uint32_t pk[kSlices][4];
#pragma unroll
      for (int t = 0; t < kSlices; ++t) pk[t][0] = pk[t][1] = pk[t][2] = pk[t][3] = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        uint32_t sl[kSlices];
        slice8(x[e], fb, sl, neg);
#pragma unroll
        for (int t = 0; t < kSlices; ++t) pk[t][e >> 1] |= sl[t] << (16 * (e & 1));
      }
#pragma unroll
      for (int t = 0; t < kSlices; ++t)
        *reinterpret_cast<uint4*>(sB + t * kBSliceBytes + (np >> 3) * 512 + q * 128 + (np & 7) * 16) =
            make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      // descriptors differ only in their address field (address / 16 < 2^14 in shared memory)
      const uint64_t ad0 = make_desc(smem_u32(sA), 128, 512), bd0 = make_desc(smem_u32(sB), 128, 512);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
        for (int s = 0; s < kGroups; ++s) {
#pragma unroll
          for (int i = 0; i <= s; ++i) {
            const uint64_t ad = ad0 + (uint64_t)((i * kASliceBytes + kk * 256) >> 4);
            const uint64_t bd = bd0 + (uint64_t)(((s - i) * kBSliceBytes + kk * 256) >> 4);
            const uint32_t acc = (ch > 0 || kk > 0 || i > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                :: "r"(tmem + (uint32_t)(s * kNr)), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&bar_mma[st])) : "memory");
      s_last = ch;
    }
  }
  __syncthreads();
  // wait for the last committed chunk (its commit covers every earlier MMA of the block)
  if (tid == 0 && s_last >= 0) {
    const int lc = s_last;
    const uint32_t bar = smem_u32(&bar_mma[lc & 1]);
    const uint32_t par = (uint32_t)((lc >> 1) & 1);
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
    if (s_fail) atomicOr(a.status, ST_TIMEOUT);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");

  if (!s_fail) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows r0 + 32 (w % 4) + lane) and
    // the complex columns 16 (w / 4) .. + 15 of the tile
    const int er = r0 + 32 * (warp & 3) + lane;
    const int eea = max(s_eh[0][er - r0], s_eh[1][er - r0]);
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
    for (int cq = 0; cq < 4; ++cq) {
      const int cb = 4 * (warp >> 2) + cq;  // 4 complex (8 real) columns
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
      double val[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const long long hi = ((((long long)gi[0][q] * 128 + gi[1][q]) * 128 + gi[2][q]) * 128) + gi[3][q];
        const long long lo = ((((long long)gi[4][q] * 128 + gi[5][q]) * 128 + gi[6][q]) * 128) + gi[7][q];
        // T = hi 2^28 + lo (|hi|, |lo| < 2^45.01): exact in int64 and rounded once when
        // |hi| < 2^34, else two exact conversions joined by one rounded fma
        val[q] = (hi > -(1ll << 34) && hi < (1ll << 34)) ? (double)(hi * (1ll << 28) + lo)
                                                          : fma((double)hi, 268435456.0, (double)lo);
      }
      if (er < m) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int c = cb * 4 + cc, col = c0 + c;
          if (col >= n) continue;
          const int fb = s_fexp[c];
          // times 2^(e_i + f_c - 2107): an integer addition to the exponent field while the
          // result stays normal, else a multiplication
          const int E = eea + fb - 2107;
          double2 p;
          if (eea == 0 || fb == 0) {
            p = make_double2(0.0, 0.0);
          } else {
            p.x = scale2(val[2 * cc], E);
            p.y = scale2(val[2 * cc + 1], E);
          }
          const double2 o = old4[cc];
          double2* cp = C + er + (long long)col * jb.ldc;
          if (a.mode == ZGEMM_SET) *cp = p;  // the mode is uniform over the launch
          else if (a.mode == ZGEMM_SUB) *cp = make_double2(o.x - p.x, o.y - p.y);
          else *cp = make_double2(o.x + p.x, o.y + p.y);
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
int zgemm_tc_max_k() { return 4 * kChunkK; }

cudaError_t launch_zgemm_tc(const ZgemmLaunch& a_in, cudaStream_t s) {
  if (a_in.ntiles <= 0) return cudaSuccess;
  ZgemmLaunch a = a_in;
  a.wait_ns = g_zgemm_wait_ns;
  a.probe_timeout = g_zgemm_probe;
  const int smem = 2 * kStageBytes;
  cudaError_t e = cudaFuncSetAttribute(zgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  zgemm_tc_kernel<<<a.ntiles, kThreads, smem, s>>>(a);
  symhss::count_launches(1);
  return cudaGetLastError();
}

}  // namespace symhss
