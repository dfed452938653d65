// Small batched operations of the factorisation and solve (Sec. 4.2):
// interpolation bases, R * X, small GEMMs (Atilde R g, f~ - Atilde y, g - X z),
// block copies (parent diagonal-block assembly), leaf gather / scatter and the
// plane-wave right-hand side.
#include <algorithm>

#include "common.cuh"

namespace symhss {

namespace {

constexpr int kOpsThreads = 256;

template <typename CT> __device__ __forceinline__ CT* bl_out(const BasisLaunch& a);
template <> __device__ __forceinline__ double2* bl_out<double2>(const BasisLaunch& a) { return a.out; }
template <> __device__ __forceinline__ float2* bl_out<float2>(const BasisLaunch& a) { return a.out32; }
template <typename CT> __device__ __forceinline__ const CT* bl_in(const BasisLaunch& a);
template <> __device__ __forceinline__ const double2* bl_in<double2>(const BasisLaunch& a) { return a.in; }
template <> __device__ __forceinline__ const float2* bl_in<float2>(const BasisLaunch& a) { return a.in32; }

// out[q[j], c] += in[col0 + j, c] (skeleton rows), out[q[r + i], c] += sum_j T[j, i] in[col0 + j, c]
// (the other active rows): out += L in with L = R^T in the diagonal-block ordering; every row
// of the box's block belongs to exactly one part's list, so each is updated by one thread
__global__ void __launch_bounds__(kOpsThreads) apply_l_kernel(const BasisLaunch a) {
  const BasisJob jb = a.jobs[blockIdx.x];
  const double2* in = a.in + jb.in_off;
  double2* out = a.out + jb.out_off;
  for (int h = 0; h < 2; ++h) {
    const BasisPart pt = jb.part[h];
    const int* q = a.q + pt.q_off;
    const double2* T = a.T + pt.t_off;
    const long long cnt = (long long)pt.n * jb.ncols;
    for (long long e = threadIdx.x + (long long)blockIdx.y * blockDim.x; e < cnt;
         e += (long long)blockDim.x * gridDim.y) {
      const int row = (int)(e % pt.n);  // position among the part's pivoted active unknowns
      const int c = (int)(e / pt.n);
      const double2* ic = in + (long long)c * jb.ld_in + pt.col0;
      double2 s;
      if (row < pt.r) {
        s = ic[row];
      } else {
        const int i = row - pt.r;
        s = make_double2(0.0, 0.0);
        for (int j = 0; j < pt.r; ++j) s = cfma(T[j + (long long)i * pt.r], ic[j], s);
      }
      double2* o = out + q[row] + (long long)c * jb.ld_out;
      *o = cadd(*o, s);
    }
  }
}

__global__ void narrow_kernel(const double2* src, float2* dst, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dst[e] = make_float2((float)src[e].x, (float)src[e].y);
}

__global__ void widen_kernel(const float2* src, double2* dst, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dst[e] = make_double2((double)src[e].x, (double)src[e].y);
}

__global__ void axpby_kernel(const double2* x, double2* y, long long n, double a, double b) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = make_double2(fma(a, x[e].x, b * y[e].x), fma(a, x[e].y, b * y[e].y));
}

// dense R^T in the diagonal-block ordering: column col0 + j holds 1 at q[j] and
// T[j, i] at q[r + i]
template <typename CT>
__global__ void __launch_bounds__(kOpsThreads) basis_dense_kernel(const BasisLaunch a) {
  const BasisJob jb = a.jobs[blockIdx.x];
  CT* out = bl_out<CT>(a) + jb.out_off;
  const long long total = (long long)jb.size * jb.k;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) out[e] = make_c<CT>(0.0, 0.0);
  __syncthreads();
  for (int h = 0; h < 2; ++h) {
    const BasisPart pt = jb.part[h];
    const int* q = a.q + pt.q_off;
    const double2* T = a.T + pt.t_off;
    const int nr = pt.n - pt.r;
    const long long cnt = (long long)pt.r * (nr + 1);
    for (long long e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int j = (int)(e % pt.r);
      const int i = (int)(e / pt.r);  // 0: skeleton entry, 1..nr: T row
      const int col = pt.col0 + j;
      if (i == 0) out[q[j] + (long long)col * jb.size] = make_c<CT>(1.0, 0.0);
      else out[q[pt.r + i - 1] + (long long)col * jb.size] = to_c<CT>(T[j + (long long)(i - 1) * pt.r]);
    }
  }
}

// out[col0 + j, c] = in[q[j], c] + sum_i T[j, i] in[q[r + i], c]
template <typename CT>
__global__ void __launch_bounds__(kOpsThreads) apply_r_kernel(const BasisLaunch a) {
  const BasisJob jb = a.jobs[blockIdx.x];
  const CT* in = bl_in<CT>(a) + jb.in_off;
  CT* out = bl_out<CT>(a) + jb.out_off;
  for (int h = 0; h < 2; ++h) {
    const BasisPart pt = jb.part[h];
    const int* q = a.q + pt.q_off;
    const double2* T = a.T + pt.t_off;
    const int nr = pt.n - pt.r;
    const long long cnt = (long long)pt.r * jb.ncols;
    for (long long e = threadIdx.x + (long long)blockIdx.y * blockDim.x; e < cnt;
         e += (long long)blockDim.x * gridDim.y) {
      const int j = (int)(e % pt.r);
      const int c = (int)(e / pt.r);
      const CT* ic = in + (long long)c * jb.ld_in;
      CT s0 = ic[q[j]], s1 = make_c<CT>(0.0, 0.0);  // two partial sums: half the dependency chain
      int i = 0;
      for (; i + 1 < nr; i += 2) {
        s0 = cfma(to_c<CT>(T[j + (long long)i * pt.r]), ic[q[pt.r + i]], s0);
        s1 = cfma(to_c<CT>(T[j + (long long)(i + 1) * pt.r]), ic[q[pt.r + i + 1]], s1);
      }
      if (i < nr) s0 = cfma(to_c<CT>(T[j + (long long)i * pt.r]), ic[q[pt.r + i]], s0);
      out[pt.col0 + j + (long long)c * jb.ld_out] = cadd(s0, s1);
    }
  }
}

// C = alpha A B + beta C; a 2-D grid of 16x16 output tiles per job
__global__ void __launch_bounds__(256) gemm_kernel(const GemmLaunch a) {
  __shared__ double2 as[16][17];
  __shared__ double2 bs[16][17];
  const GemmJob jb = a.jobs[blockIdx.x];
  const int tiles_m = (jb.m + 15) / 16, tiles_n = (jb.n + 15) / 16;
  const double2* A = a.A + jb.a_off;
  const double2* B = a.B + jb.b_off;
  double2* C = a.C + jb.c_off;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int tile = blockIdx.y; tile < tiles_m * tiles_n; tile += gridDim.y) {
    const int i0 = (tile % tiles_m) * 16, j0 = (tile / tiles_m) * 16;
    double2 acc = make_double2(0.0, 0.0);
    for (int l0 = 0; l0 < jb.k; l0 += 16) {
      const int ai = i0 + tx, al = l0 + ty;
      as[ty][tx] = (ai < jb.m && al < jb.k) ? A[ai + (long long)al * jb.lda] : make_double2(0.0, 0.0);
      const int bl = l0 + tx, bj = j0 + ty;
      bs[ty][tx] = (bl < jb.k && bj < jb.n) ? B[bl + (long long)bj * jb.ldb] : make_double2(0.0, 0.0);
      __syncthreads();
#pragma unroll
      for (int l = 0; l < 16; ++l) acc = cfma(as[l][tx], bs[ty][l], acc);
      __syncthreads();
    }
    const int i = i0 + tx, j = j0 + ty;
    if (i < jb.m && j < jb.n) {
      double2* c = C + i + (long long)j * jb.ldc;
      double2 v = make_double2(jb.alpha * acc.x, jb.alpha * acc.y);
      if (jb.beta != 0.0) v = make_double2(v.x + jb.beta * c->x, v.y + jb.beta * c->y);
      *c = v;
    }
  }
}

// The same product for narrow B (at most kGemvCols columns: the solve phase and the
// refinement matvecs carry one or a few right-hand sides): a block takes 32 rows of C, lane =
// row, and its 8 warps split the inner dimension; the partial sums meet in shared memory.
// Every FP64 instruction works on 32 useful lanes, where 16 x 16 output tiles would leave
// all but one tile column idle.
constexpr int kGemvCols = 4;
__global__ void __launch_bounds__(256) gemv_kernel(const GemmLaunch a) {
  __shared__ double2 part[8][kGemvCols][32];
  const GemmJob jb = a.jobs[blockIdx.x];
  const int i0 = blockIdx.y * 32;
  if (i0 >= jb.m || jb.n > kGemvCols) return;  // uniform per block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = i0 + lane, nc = jb.n;
  const int kper = (jb.k + 7) / 8;
  const int l0 = warp * kper, l1 = min(jb.k, l0 + kper);
  const double2* A = a.A + jb.a_off;
  const double2* B = a.B + jb.b_off;
  double2 acc[kGemvCols];
#pragma unroll
  for (int c = 0; c < kGemvCols; ++c) acc[c] = make_double2(0.0, 0.0);
  if (i < jb.m) {
    for (int l = l0; l < l1; ++l) {
      const double2 av = A[i + (long long)l * jb.lda];
#pragma unroll
      for (int c = 0; c < kGemvCols; ++c)
        if (c < nc) acc[c] = cfma(av, B[l + (long long)c * jb.ldb], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < kGemvCols; ++c) part[warp][c][lane] = acc[c];
  __syncthreads();
  if (warp < nc && i < jb.m) {  // warp c sums column c over the 8 slices
    double2 v = make_double2(0.0, 0.0);
#pragma unroll
    for (int w = 0; w < 8; ++w) v = cadd(v, part[w][warp][lane]);
    double2* c = a.C + jb.c_off + i + (long long)warp * jb.ldc;
    double2 r = make_double2(jb.alpha * v.x, jb.alpha * v.y);
    if (jb.beta != 0.0) r = make_double2(r.x + jb.beta * c->x, r.y + jb.beta * c->y);
    *c = r;
  }
}

template <typename CT>
__global__ void __launch_bounds__(kOpsThreads) copy_kernel(const CT* src, CT* dst,
                                                           const CopyJob* jobs) {
  const CopyJob jb = jobs[blockIdx.x];
  const long long total = (long long)jb.rows * jb.cols;
  for (long long e = threadIdx.x + (long long)blockIdx.y * blockDim.x; e < total;
       e += (long long)blockDim.x * gridDim.y) {
    const int i = (int)(e % jb.rows), j = (int)(e / jb.rows);
    CT v;
    if (jb.src_off >= 0) v = src[jb.src_off + i + (long long)j * jb.lds];
    else v = make_c<CT>(i == j ? 1.0 : 0.0, 0.0);
    if (jb.trans) dst[jb.dst_off + j + (long long)i * jb.ldd] = v;
    else dst[jb.dst_off + i + (long long)j * jb.ldd] = v;
  }
}

__global__ void __launch_bounds__(kOpsThreads) leaf_gather_kernel(const double2* f, long long ldf, double2* g,
                                                                  const LeafJob* jobs, int nrhs) {
  const LeafJob jb = jobs[blockIdx.x];
  const int size = 2 * jb.len;
  for (int e = threadIdx.x; e < size * nrhs; e += blockDim.x) {
    const int i = e % size, c = e / size;
    const long long src = jb.base + (i < jb.len ? jb.begin + i : jb.n + jb.begin + (i - jb.len));
    g[jb.off + i + (long long)c * size] = f[src + (long long)c * ldf];
  }
}

__global__ void __launch_bounds__(kOpsThreads) leaf_scatter_kernel(const double2* g, double2* x, long long ldx,
                                                                   const LeafJob* jobs, int nrhs) {
  const LeafJob jb = jobs[blockIdx.x];
  const int size = 2 * jb.len;
  for (int e = threadIdx.x; e < size * nrhs; e += blockDim.x) {
    const int i = e % size, c = e / size;
    const long long dst = jb.base + (i < jb.len ? jb.begin + i : jb.n + jb.begin + (i - jb.len));
    x[dst + (long long)c * ldx] = g[jb.off + i + (long long)c * size];
  }
}

__global__ void plane_wave_kernel(const PointTable t, const WaveJob* jobs, double ca, double sa, int scaled,
                                  double2* rhs) {
  const WaveJob jb = jobs[blockIdx.y];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= jb.n) return;
  const int i = jb.node0 + j;
  double sn, cs;
  sincos(jb.k0 * (t.x[i] * ca + t.y[i] * sa), &sn, &cs);
  const double2 uin = make_double2(cs, sn);
  const double dn = jb.k0 * (t.nx[i] * ca + t.ny[i] * sa);
  const double2 dudn = make_double2(-dn * sn, dn * cs);  // i k0 (nu.dir) u_in
  const double sc = scaled ? t.w[i] : 1.0;
  double2* r = rhs + jb.vec0;
  const double2 r1 = cadd(cmul(jb.a1, uin), cmul(jb.b1, dudn));
  const double2 r2 = cadd(cmul(jb.a2, uin), cmul(jb.b2, dudn));
  r[j] = make_double2(sc * r1.x, sc * r1.y);
  r[jb.n + j] = make_double2(sc * r2.x, sc * r2.y);
}

}  // namespace

cudaError_t launch_basis_dense(const BasisLaunch& a, cudaStream_t s) {
  if (a.njobs <= 0) return cudaSuccess;
  if (a.out32) basis_dense_kernel<float2><<<a.njobs, kOpsThreads, 0, s>>>(a);
  else basis_dense_kernel<double2><<<a.njobs, kOpsThreads, 0, s>>>(a);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_apply_r(const BasisLaunch& a, cudaStream_t s) {
  if (a.njobs <= 0) return cudaSuccess;
  // blocks per job so that even the few boxes of the top levels spread over every SM
  const int per_job = std::max(4, std::min(64, (4 * device_sm_count() + a.njobs - 1) / a.njobs));
  dim3 grid(a.njobs, per_job);
  if (a.out32) apply_r_kernel<float2><<<grid, kOpsThreads, 0, s>>>(a);
  else apply_r_kernel<double2><<<grid, kOpsThreads, 0, s>>>(a);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gemm(const GemmLaunch& a, cudaStream_t s) {
  if (a.njobs <= 0) return cudaSuccess;
  if (a.max_m > 0 && a.max_n > 0 && a.max_n <= kGemvCols) {
    gemv_kernel<<<dim3(a.njobs, (a.max_m + 31) / 32), 256, 0, s>>>(a);
    symhss::count_launches(1);
    return cudaGetLastError();
  }
  dim3 grid(a.njobs, 8);
  gemm_kernel<<<grid, 256, 0, s>>>(a);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_copy_blocks(const double2* src, double2* dst, const CopyJob* jobs, int njobs,
                               cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  dim3 grid(njobs, 4);
  copy_kernel<double2><<<grid, kOpsThreads, 0, s>>>(src, dst, jobs);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_copy_blocks32(const float2* src, float2* dst, const CopyJob* jobs, int njobs, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  dim3 grid(njobs, 4);
  copy_kernel<float2><<<grid, kOpsThreads, 0, s>>>(src, dst, jobs);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_apply_l(const BasisLaunch& a, cudaStream_t s) {
  if (a.njobs <= 0) return cudaSuccess;
  dim3 grid(a.njobs, 4);
  apply_l_kernel<<<grid, kOpsThreads, 0, s>>>(a);
  symhss::count_launches(1);
  return cudaGetLastError();
}

static int elementwise_blocks(long long n) {
  const long long b = (n + 255) / 256;
  const long long cap = 16LL * device_sm_count();
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

cudaError_t launch_narrow(const double2* src, float2* dst, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  narrow_kernel<<<elementwise_blocks(n), 256, 0, s>>>(src, dst, n);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_widen(const float2* src, double2* dst, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  widen_kernel<<<elementwise_blocks(n), 256, 0, s>>>(src, dst, n);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_axpby(const double2* x, double2* y, long long n, double a, double b, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  axpby_kernel<<<elementwise_blocks(n), 256, 0, s>>>(x, y, n, a, b);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_leaf_gather(const double2* f, long long ldf, double2* g, const LeafJob* jobs, int njobs,
                               int nrhs, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  leaf_gather_kernel<<<njobs, kOpsThreads, 0, s>>>(f, ldf, g, jobs, nrhs);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_leaf_scatter(const double2* g, double2* x, long long ldx, const LeafJob* jobs, int njobs,
                                int nrhs, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  leaf_scatter_kernel<<<njobs, kOpsThreads, 0, s>>>(g, x, ldx, jobs, nrhs);
  symhss::count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_plane_wave(const PointTable& t, const WaveJob* jobs, int njobs, int max_n, double angle,
                              int scaled, double2* rhs, cudaStream_t s) {
  if (njobs <= 0 || max_n <= 0) return cudaSuccess;
  dim3 grid((max_n + 255) / 256, njobs);
  plane_wave_kernel<<<grid, 256, 0, s>>>(t, jobs, cos(angle), sin(angle), scaled, rhs);
  symhss::count_launches(1);
  return cudaGetLastError();
}

}  // namespace symhss
