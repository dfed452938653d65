// Randomized row sketch of the proxy matrices, Y = Omega M (s x n), computed on the
// 5th-generation tensor cores (tcgen05) to FP64 accuracy.  The column ID is then
// taken of Y instead of M (randomized ID, Halko-Martinsson-Tropp): Y has s =
// rank estimate + oversampling rows instead of the m rows of M.
//
// Exact splitting.  Omega is a Rademacher (+-1) matrix, exact in bf16, drawn from
// the counter-based generator splitmix64(seed ^ job * C1 ^ row * C2 ^ col) (sign of
// the top bit).  M is complex FP64; the real and imaginary parts form the 2n real
// columns of B = [Re M | Im M].  Each column c of B is scaled by its exponent e_c
// (|B(:, c)| < 2^e_c) and cut into 7 slices of 8 bits by integer operations on the
// FP64 bit pattern:  B(k, c) = sign * sum_t d_t(k, c) 2^(e_c - 8(t+1)), 0 <= d_t <= 255,
// dropping only bits below 2^(e_c - 56).  Every d_t is exact in bf16, every product
// Omega * d_t is an integer of at most 8 bits, and a sum over m <= 65536 rows stays
// below 2^24, so each slice product Omega S_t is exact in the FP32 accumulator.  Y is
// then sum_t 2^(e_c - 8(t+1)) (Omega S_t) in FP64.
//
// GEMM.  One thread block computes a 128-row x 32-column tile of Y for all 7 slices
// at once: the MMA is M = 128, N = 224 (7 slices x 32 columns), K = 16, bf16 x bf16
// -> FP32, accumulator in tensor memory (256 columns).  Per K-chunk of 64 rows of M
// the block writes its Omega chunk into shared memory and one bulk asynchronous copy
// brings the 28 KB of slices (stored in global memory already in the core-matrix
// order the MMA reads), then one elected thread issues 4 MMAs and commits them to an
// mbarrier.  Every wait is bounded in time (%globaltimer, kWaitNs by default).  On a
// timeout the block records ST_TIMEOUT, then waits once more (bounded by kWaitNs) for the
// work it may still have in flight -- the bulk copy into shared memory or the MMAs writing
// tensor memory -- and only then frees its tensor memory and exits, so no late write can
// land in shared or tensor memory that another block owns by then.
//
// Recombination.  Each slice product v_t = (Omega S_t)(i, c) is an integer below 2^24 held
// exactly in FP32.  The epilogue converts the seven to int32 and forms two exact int64
// partial sums, hi = v0 2^16 + v1 2^8 + v2 (< 2^41) and lo = v3 2^24 + v4 2^16 + v5 2^8 + v6
// (< 2^49), so Y(i, c) = hi 2^(e_c - 24) + lo 2^(e_c - 56) with one FP64 rounding.
#include <stdint.h>

#include "common.cuh"

namespace symhss {

namespace {

constexpr int kSlices = 7;
constexpr int kMTile = 128;        // rows of Y per block (MMA M)
constexpr int kNCols = 32;         // columns of B per block (per slice)
constexpr int kN = kSlices * kNCols;  // MMA N = 224
constexpr int kKChunk = 64;        // rows of M per pipeline step
constexpr int kTmemCols = 256;     // power of two >= kN
constexpr int kBlockBytes = kSlices * kNCols * kKChunk * 2;  // 28672: one (column block, K-chunk) of slices
constexpr int kABytes = kMTile * kKChunk * 2;                // 16384: Omega chunk
constexpr int kThreads = 128;
constexpr long long kWaitNs = 200ll * 1000 * 1000;  // 200 ms per wait

long long g_wait_ns = kWaitNs;

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// +-1 entry of Omega for (job stream id, row i of Y, row k of M)
__device__ __forceinline__ bool omega_negative(uint64_t seed, uint64_t stream, int i, int k) {
  const uint64_t h = splitmix64(seed ^ (stream * 0xD1B54A32D192ED03ull) ^ ((uint64_t)i * 0x8CB92BA72F3D8DD7ull) ^
                                (uint64_t)k);
  return (h >> 63) != 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// no-swizzle K-major shared-memory matrix descriptor (core matrices of 8 rows x 16 bytes)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // fixed 0b001 in bits 46-48
  return d;                // base offset 0, relative LBO, no swizzle
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

// wait for phase `parity` of an mbarrier for at most limit_ns nanoseconds (at least one try)
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

// ---- slicing: B = [Re M | Im M] -> 7 bf16 slices in the MMA core-matrix order ----------
// one warp per complex column j of one job: column exponents, then slices of 8 rows per lane
__global__ void __launch_bounds__(256) slice_kernel(const SketchLaunch a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * 8 + warp;
  if (gw >= a.ncolwork) return;
  const SketchColWork cw = a.colwork[gw];
  const SketchJob jb = a.jobs[cw.job];
  const int j = cw.col;
  const double2* col = a.mats + jb.m_off + (long long)j * jb.ld;
  // largest biased exponent of the real and of the imaginary part
  int er = 0, ei = 0;
  for (int k = lane; k < jb.m; k += 32) {
    const double2 v = col[k];
    er = max(er, (int)((__double_as_longlong(v.x) >> 52) & 0x7FF));
    ei = max(ei, (int)((__double_as_longlong(v.y) >> 52) & 0x7FF));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    er = max(er, __shfl_xor_sync(0xffffffffu, er, o));
    ei = max(ei, __shfl_xor_sync(0xffffffffu, ei, o));
  }
  const int n2 = jb.n2pad;
  if (lane == 0) {
    a.exps[jb.exp_off + j] = er;            // column j of B (real part)
    a.exps[jb.exp_off + jb.n + j] = ei;     // column n + j of B (imaginary part)
  }
  const int nk = jb.mpad / kKChunk;
  for (int part = 0; part < 2; ++part) {
    const int c = part == 0 ? j : jb.n + j;  // column of B
    const int emax = part == 0 ? er : ei;
    const int cb = c / kNCols, cc = c % kNCols;
    const int g = cc >> 3, r = cc & 7;
    for (int grp = lane; grp < jb.mpad / 8; grp += 32) {  // 8 consecutive rows of M
      const int k0 = grp * 8;
      const int kc = k0 / kKChunk, h = (k0 % kKChunk) >> 3;
      uint32_t packed[kSlices][4];
#pragma unroll
      for (int t = 0; t < kSlices; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) packed[t][q] = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + e;
        const double x = (k < jb.m) ? (part == 0 ? col[k].x : col[k].y) : 0.0;
        const long long bits = __double_as_longlong(x);
        const int E = (int)((bits >> 52) & 0x7FF);
        uint64_t A = 0;
        if (E != 0 && emax != 0) {
          const uint64_t mant = ((uint64_t)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
          const int sh = E - emax + 3;  // A = |x| 2^(56 - e_c), e_c = emax - 1022
          A = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
        }
        const uint32_t sgn = (bits < 0) ? 0x8000u : 0u;
#pragma unroll
        for (int t = 0; t < kSlices; ++t) {
          const uint32_t d = (uint32_t)((A >> (48 - 8 * t)) & 0xFF);
          const uint32_t bf = d ? ((__float_as_uint((float)d) >> 16) | sgn) : 0u;
          packed[t][e >> 1] |= bf << (16 * (e & 1));
        }
      }
      // block (cb, kc): [t][g][h][r][8 K values]
      uint8_t* blk = a.slices + jb.slice_off + ((long long)cb * nk + kc) * kBlockBytes;
#pragma unroll
      for (int t = 0; t < kSlices; ++t) {
        uint4 v = make_uint4(packed[t][0], packed[t][1], packed[t][2], packed[t][3]);
        *reinterpret_cast<uint4*>(blk + t * 4096 + g * 1024 + h * 128 + r * 16) = v;
      }
    }
  }
  (void)n2;
}

// ---- tcgen05 GEMM + FP64 recombination ---------------------------------------------------
__global__ void __launch_bounds__(kThreads) sketch_mma_kernel(const SketchLaunch a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sa = smem;                 // Omega chunk, 16 KB
  unsigned char* sb = smem + kABytes;       // slice block, 28 KB
  __shared__ __align__(8) uint64_t bar_tx, bar_mma;
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_fail;
  const SketchTile tl = a.tiles[blockIdx.x];
  const SketchJob jb = a.jobs[tl.job];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = jb.mpad / kKChunk;
  const int row0 = tl.mtile * kMTile;

  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_tx)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_mma)));
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
  const uint32_t idesc = make_idesc(kMTile, kN);
  const uint64_t stream = (uint64_t)jb.stream_id;

  // s_fail: 0 = fine; 1 + 2 kc: the wait for chunk kc's copy expired (copy maybe in flight);
  // 2 + 2 kc: the wait for chunk kc's MMAs expired (MMAs maybe in flight)
  for (int kc = 0; kc < nk; ++kc) {
    const uint32_t parity = (uint32_t)(kc & 1);
    // slices of this K-chunk: one bulk copy
    if (tid == 0) {
      const uint8_t* src = a.slices + jb.slice_off + ((long long)tl.cb * nk + kc) * kBlockBytes;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   :: "r"(smem_u32(&bar_tx)), "r"(kBlockBytes) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   :: "r"(smem_u32(sb)), "l"(src), "r"(kBlockBytes), "r"(smem_u32(&bar_tx)) : "memory");
    }
    // Omega chunk: rows row0..row0+127 of Y, K rows kc*64..kc*64+63 of M, core-matrix order
    for (int q = tid; q < kMTile * kKChunk / 8; q += kThreads) {  // one 16-byte row of a core matrix each
      const int G = q / 64, rem = q % 64, h = rem / 8, r = rem % 8;
      const int i = row0 + G * 8 + r;
      uint32_t w[4] = {0, 0, 0, 0};
      if (i < jb.s) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = kc * kKChunk + h * 8 + e;
          uint32_t bf = 0;
          if (k < jb.m) bf = omega_negative(a.seed, stream, i, k) ? 0xBF80u : 0x3F80u;
          w[e >> 1] |= bf << (16 * (e & 1));
        }
      }
      *reinterpret_cast<uint4*>(sa + G * 1024 + h * 128 + r * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && !mbar_wait(smem_u32(&bar_tx), parity, a.wait_ns)) s_fail = 1 + 2 * kc;
    __syncthreads();
    if (s_fail) break;  // uniform: read after the barrier
    // every thread observes the completed copy before the MMAs read it
    mbar_wait(smem_u32(&bar_tx), parity, kWaitNs);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
#pragma unroll
      for (int kk = 0; kk < kKChunk / 16; ++kk) {
        const uint64_t ad = make_desc(smem_u32(sa) + kk * 256, 128, 1024);
        const uint64_t bd = make_desc(smem_u32(sb) + kk * 256, 128, 1024);
        const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&bar_mma)) : "memory");
      if (!mbar_wait(smem_u32(&bar_mma), parity, a.wait_ns)) s_fail = 2 + 2 * kc;
    }
    __syncthreads();
    if (s_fail) break;
    // every thread observes the completed MMAs before shared memory is rewritten or TMEM read
    mbar_wait(smem_u32(&bar_mma), parity, kWaitNs);
    asm volatile("tcgen05.fence::after_thread_sync;");
  }

  if (s_fail) {
    // drain: wait (bounded, default limit) for the copy or the MMAs that may be in flight
    if (tid == 0) {
      const int f = s_fail - 1;
      const uint32_t par = (uint32_t)((f >> 1) & 1);
      mbar_wait(smem_u32((f & 1) ? &bar_mma : &bar_tx), par, kWaitNs);
      atomicOr(a.status, ST_TIMEOUT);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
  }

  if (!s_fail) {
    // epilogue: warp w reads rows 32w..32w+31 (TMEM lanes); two halves of 16 columns
    const int row = row0 + warp * 32 + lane;
    double* y = reinterpret_cast<double*>(a.y + jb.y_off);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      long long hi[16], lo[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) { hi[c] = 0; lo[c] = 0; }
#pragma unroll
      for (int t = 0; t < kSlices; ++t) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * kNCols + half * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
            " [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          // exact: the FP32 accumulator holds an integer below 2^24
          const long long d = (long long)__float2int_rn(__uint_as_float(v[c]));
          if (t < 3) hi[c] = hi[c] * 256 + d;
          else lo[c] = lo[c] * 256 + d;
        }
      }
      if (row < jb.s) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int bc = tl.cb * kNCols + half * 16 + c;
          if (bc >= 2 * jb.n) continue;
          const int ec = a.exps[jb.exp_off + bc];  // biased exponent of the column's largest entry
          // slice t carries weight 2^(ec - 1022 - 8(t+1)): hi at 2^(ec - 1046), lo at 2^(ec - 1078)
          const double val = ec ? fma((double)hi[c], ldexp(1.0, ec - 1046), ldexp((double)lo[c], ec - 1078)) : 0.0;
          if (bc < jb.n) y[2 * (row + (long long)bc * jb.ldy)] = val;
          else y[2 * (row + (long long)(bc - jb.n) * jb.ldy) + 1] = val;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
}

}  // namespace

uint64_t sketch_host_splitmix64(uint64_t x) { return splitmix64(x); }

size_t sketch_slice_bytes(int mpad, int n2pad) {
  return (size_t)(n2pad / kNCols) * (mpad / kKChunk) * kBlockBytes;
}
int sketch_mpad(int m) { return ((m + kKChunk - 1) / kKChunk) * kKChunk; }
int sketch_n2pad(int n) { return ((2 * n + kNCols - 1) / kNCols) * kNCols; }

void set_sketch_wait_ns(long long ns) { g_wait_ns = ns > 0 ? ns : kWaitNs; }

cudaError_t launch_sketch(const SketchLaunch& a_in, cudaStream_t s) {
  if (a_in.ncolwork <= 0 || a_in.ntiles <= 0) return cudaSuccess;
  SketchLaunch a = a_in;
  a.wait_ns = g_wait_ns;
  slice_kernel<<<(a.ncolwork + 7) / 8, 256, 0, s>>>(a);
  symhss::count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // 112 KB of dynamic shared memory keeps at most two blocks (2 x 256 tensor-memory
  // columns) on an SM, so every tensor-memory allocation is satisfied without waiting
  const int smem = 112 * 1024;
  e = cudaFuncSetAttribute(sketch_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  sketch_mma_kernel<<<a.ntiles, kThreads, smem, s>>>(a);
  symhss::count_launches(1);
  return cudaGetLastError();
}

}  // namespace symhss
