// Stand-alone building-block entry points of the C ABI (include/symhss.h):
// the tile generator on explicit point sets, the batched column ID and the
// batched LU / solve.  They validate their arguments, allocate the small job
// arrays they need, launch the same kernels the solver uses, and synchronise
// the stream before returning.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

using namespace symhss;

namespace {
std::atomic<long long> g_launches{0};
}  // namespace

void symhss::count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int symhss::device_sm_count() {
  static std::atomic<int> cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 148;
  if (dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
  if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

namespace {

struct TmpBuf {
  void* p = nullptr;
  ~TmpBuf() { if (p) cudaFree(p); }
  cudaError_t alloc(size_t b) { return cudaMalloc(&p, b ? b : 16); }
};

int cerr(cudaError_t e) { return e == cudaErrorMemoryAllocation ? SYMHSS_ERR_NOMEM : SYMHSS_ERR_CUDA; }

#define CKE(call)                                  \
  do {                                             \
    cudaError_t _e = (call);                       \
    if (_e != cudaSuccess) return cerr(_e);        \
  } while (0)

int status_code(int st) {
  if (st & ST_BAD_INDEX) return SYMHSS_ERR_DEVICE;
  if (st & ST_SINGULAR) return SYMHSS_ERR_SINGULAR;
  if (st & ST_TIMEOUT) return SYMHSS_ERR_TIMEOUT;
  if (st) return SYMHSS_ERR_DEVICE;
  return SYMHSS_OK;
}

}  // namespace

// Central differences of order 2m on a periodic sequence, unit spacing, with the closed-form
// weights  a_j = (-1)^(j+1) c_j / j  (first derivative, on f[i+j] - f[i-j]) and
// b_j = 2 (-1)^(j+1) c_j / j^2  (second derivative, on f[i+j] + f[i-j]; centre -2 sum b_j),
// c_j = (m!)^2 / ((m-j)! (m+j)!) = prod_{t=1..j} (m-j+t) / (m+t).
void symhss::speed_terms(const double* w, int n, double* out) {
  const int m = std::max(0, std::min(8, (n - 1) / 2));
  if (m == 0) {
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    return;
  }
  double a[9] = {0}, b[9] = {0}, b0 = 0.0;
  for (int j = 1; j <= m; ++j) {
    double c = 1.0;
    for (int t = 1; t <= j; ++t) c *= (double)(m - j + t) / (double)(m + t);
    const double sg = (j % 2 == 1) ? 1.0 : -1.0;
    a[j] = sg * c / j;
    b[j] = 2.0 * sg * c / ((double)j * j);
    b0 -= 2.0 * b[j];
  }
  const double inv2pi = 1.0 / (2.0 * 3.141592653589793238462643383279502884);
  for (int i = 0; i < n; ++i) {
    double d1 = 0.0, d2 = b0 * w[i];
    for (int j = 1; j <= m; ++j) {
      const double fp = w[(i + j) % n], fm = w[((i - j) % n + n) % n];
      d1 += a[j] * (fp - fm);
      d2 += b[j] * (fp + fm);
    }
    const double l1 = d1 / w[i], l2 = d2 / w[i];
    out[i] = (l2 / 6.0 - 0.25 * l1 * l1) * inv2pi;
  }
}

namespace {

bool points_ok(const symhss_points* p) {
  return p && p->n >= 0 && (p->n == 0 || (p->x && p->y && p->nx && p->ny && p->w && p->kappa && p->id));
}

}  // namespace

extern "C" {

long long symhss_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int symhss_set_wait_limit_ns(long long ns) {
  symhss::set_sketch_wait_ns(ns);
  symhss::set_zgemm_wait_ns(ns);
  return SYMHSS_OK;
}

int symhss_set_timeout_probe(int on) {
  symhss::set_zgemm_timeout_probe(on);
  return SYMHSS_OK;
}

int symhss_zgemm(const void* A, int lda, long long strideA, const void* B, int ldb, long long strideB, void* C,
                 int ldc, long long strideC, int m, int n, int k, int batch, int mode, void* stream) {
  if (m < 0 || n < 0 || k < 0 || batch < 0 || mode < 0 || mode > 2) return SYMHSS_ERR_INVALID;
  if (m == 0 || n == 0 || batch == 0) return SYMHSS_OK;
  if (!C || ldc < m || strideC < (long long)ldc * n) return SYMHSS_ERR_INVALID;
  if (k > 0 && (!A || !B || lda < m || ldb < k || strideA < (long long)lda * k || strideB < (long long)ldb * n))
    return SYMHSS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (k == 0) {
    if (mode != ZGEMM_SET) return SYMHSS_OK;
    for (int b = 0; b < batch; ++b)
      CKE(cudaMemset2DAsync(reinterpret_cast<double2*>(C) + strideC * b, (size_t)ldc * sizeof(double2), 0,
                            (size_t)m * sizeof(double2), n, s));
    CKE(cudaStreamSynchronize(s));
    return SYMHSS_OK;
  }
  const int TM = zgemm_tc_tile_rows(), TN = zgemm_tc_tile_cols(), KM = zgemm_tc_max_k();
  const int mt = (m + TM - 1) / TM, nt = (n + TN - 1) / TN;
  std::vector<ZgemmTile> tiles;
  for (int b = 0; b < batch; ++b)
    for (int i = 0; i < mt; ++i)
      for (int j = 0; j < nt; ++j) tiles.push_back(ZgemmTile{b, i, j});
  const int nchunk = (k + KM - 1) / KM;
  const size_t o_jobs = 0;
  const size_t o_tiles = ((size_t)batch * nchunk * sizeof(ZgemmJob) + 255) & ~size_t(255);
  const size_t o_status = o_tiles + ((tiles.size() * sizeof(ZgemmTile) + 255) & ~size_t(255));
  const size_t total = o_status + 256;
  std::vector<char> host(total, 0);
  ZgemmJob* jobs = reinterpret_cast<ZgemmJob*>(host.data() + o_jobs);
  for (int c = 0; c < nchunk; ++c)
    for (int b = 0; b < batch; ++b) {
      ZgemmJob& j = jobs[(size_t)c * batch + b];
      const int k0 = c * KM;
      j.a_off = strideA * b + (long long)k0 * lda;
      j.b_off = strideB * b + k0;
      j.c_off = strideC * b;
      j.m = m; j.n = n; j.k = std::min(KM, k - k0);
      j.lda = lda; j.ldb = ldb; j.ldc = ldc;
    }
  std::memcpy(host.data() + o_tiles, tiles.data(), tiles.size() * sizeof(ZgemmTile));
  TmpBuf meta;
  CKE(meta.alloc(total));
  CKE(cudaMemcpyAsync(meta.p, host.data(), total, cudaMemcpyHostToDevice, s));
  char* d = reinterpret_cast<char*>(meta.p);
  ZgemmLaunch a;
  a.A = reinterpret_cast<const double2*>(A);
  a.B = reinterpret_cast<const double2*>(B);
  a.C = reinterpret_cast<double2*>(C);
  a.tiles = reinterpret_cast<const ZgemmTile*>(d + o_tiles);
  a.ntiles = (int)tiles.size();
  a.status = reinterpret_cast<int*>(d + o_status);
  a.wait_ns = 0;
  a.njobs = batch;
  a.mtiles = mt;
  a.ntiles_c = nt;
  TmpBuf img;  // slice images, reused by the chunks of k one after another on the stream
  a.img_bytes = zgemm_img_bytes(batch, mt, nt);
  CKE(img.alloc((size_t)a.img_bytes));
  a.img = reinterpret_cast<unsigned char*>(img.p);
  // chunks of k in order on the stream: the first sets (or updates) C, the rest accumulate
  for (int c = 0; c < nchunk; ++c) {
    a.jobs = reinterpret_cast<const ZgemmJob*>(d + o_jobs) + (size_t)c * batch;
    a.mode = (c == 0) ? mode : (mode == ZGEMM_SUB ? ZGEMM_SUB : ZGEMM_ADD);
    CKE(launch_zgemm_tc(a, s));
  }
  int st = 0;
  CKE(cudaMemcpyAsync(&st, a.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKE(cudaStreamSynchronize(s));
  return status_code(st);
}

int symhss_speed_terms(const double* w, int n, double* s) {
  if (n < 1 || !w || !s) return SYMHSS_ERR_INVALID;
  for (int i = 0; i < n; ++i)
    if (!(w[i] > 0) || !std::isfinite(w[i])) return SYMHSS_ERR_INVALID;
  symhss::speed_terms(w, n, s);
  return SYMHSS_OK;
}

int symhss_hankel01(const double* x, int n, void* out, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return SYMHSS_ERR_INVALID;
  if (n == 0) return SYMHSS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  CKE(launch_hankel(x, n, reinterpret_cast<double2*>(out), s));
  CKE(cudaStreamSynchronize(s));
  return SYMHSS_OK;
}

int symhss_pivot_reciprocal(const void* a, int n, void* out, void* stream) {
  if (n < 0 || (n > 0 && (!a || !out))) return SYMHSS_ERR_INVALID;
  if (n == 0) return SYMHSS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  CKE(launch_pivot_reciprocal(reinterpret_cast<const double2*>(a), n, reinterpret_cast<double2*>(out), s));
  CKE(cudaStreamSynchronize(s));
  return SYMHSS_OK;
}

int symhss_kernel_block(const symhss_params* prm, const symhss_points* obs, const int* obs_eq,
                        const symhss_points* src, const int* src_comp, int scaled, void* out, int ld,
                        void* stream) {
  if (!prm || !points_ok(obs) || !points_ok(src) || !out) return SYMHSS_ERR_INVALID;
  if (!(prm->k0 > 0) || !(prm->k1 > 0) || !std::isfinite(prm->eps0) || !std::isfinite(prm->eps1))
    return SYMHSS_ERR_INVALID;
  if (!(prm->eps0 != 0.0) || !(prm->eps1 != 0.0)) return SYMHSS_ERR_INVALID;
  if (prm->formulation != SYMHSS_MULLER && prm->formulation != SYMHSS_PMCHWT && prm->formulation != SYMHSS_BM)
    return SYMHSS_ERR_INVALID;
  if (ld < obs->n || ld < 1) return SYMHSS_ERR_INVALID;
  if ((obs->n > 0 && !obs_eq) || (src->n > 0 && !src_comp)) return SYMHSS_ERR_INVALID;
  if (obs->n == 0 || src->n == 0) return SYMHSS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int m = obs->n, n = src->n;
  // equation / component labels live on the device: fetch them to build the slot lists
  std::vector<int> eq(m), comp(n);
  CKE(cudaMemcpyAsync(eq.data(), obs_eq, m * sizeof(int), cudaMemcpyDeviceToHost, s));
  CKE(cudaMemcpyAsync(comp.data(), src_comp, n * sizeof(int), cudaMemcpyDeviceToHost, s));
  CKE(cudaStreamSynchronize(s));
  std::vector<int> tp(m), ts0(m), ts1(m), lp(n), ls0(n), ls1(n);
  for (int i = 0; i < m; ++i) {
    if (eq[i] != 0 && eq[i] != 1) return SYMHSS_ERR_INVALID;
    tp[i] = i; ts0[i] = eq[i] == 0 ? i : -1; ts1[i] = eq[i] == 1 ? i : -1;
  }
  for (int j = 0; j < n; ++j) {
    if (comp[j] != 0 && comp[j] != 1) return SYMHSS_ERR_INVALID;
    lp[j] = j; ls0[j] = comp[j] == 0 ? j : -1; ls1[j] = comp[j] == 1 ? j : -1;
  }
  TileJob jb;
  jb.tp_off = 0; jb.n_tp = m; jb.lp_off = 0; jb.n_lp = n; jb.out_off = 0; jb.ld = ld;
  jb.flags = scaled ? 0 : TILE_UNSCALED;
  jb.prm = 0;
  jb.pad_ = 0;
  std::vector<TileChunk> ch;
  for (int a = 0; a < m; a += TILE_T)
    for (int b = 0; b < n; b += TILE_L) ch.push_back(TileChunk{0, a, b, TILE_L});
  const size_t ints = 3 * (size_t)m + 3 * (size_t)n;
  TmpBuf buf;
  const size_t bytes = ints * sizeof(int) + sizeof(TileJob) + ch.size() * sizeof(TileChunk) + sizeof(int) +
                       sizeof(KernelParams) + 128;
  CKE(buf.alloc(bytes));
  std::vector<char> host(bytes, 0);
  char* hp = host.data();
  size_t off = 0;
  auto put = [&](const void* src_, size_t b) { std::memcpy(hp + off, src_, b); size_t o = off; off += b; return o; };
  const size_t o1 = put(tp.data(), m * 4), o2 = put(ts0.data(), m * 4), o3 = put(ts1.data(), m * 4);
  const size_t o4 = put(lp.data(), n * 4), o5 = put(ls0.data(), n * 4), o6 = put(ls1.data(), n * 4);
  off = (off + 15) & ~size_t(15);
  const size_t o7 = put(&jb, sizeof(jb));
  const size_t o8 = put(ch.data(), ch.size() * sizeof(TileChunk));
  off = (off + 15) & ~size_t(15);
  const KernelParams kp = make_kernel_params(*prm);
  const size_t o10 = put(&kp, sizeof(kp));
  const size_t o9 = off;
  CKE(cudaMemcpyAsync(buf.p, hp, bytes, cudaMemcpyHostToDevice, s));
  char* d = reinterpret_cast<char*>(buf.p);
  TileLaunch a;
  a.tpts = PointTable{obs->x, obs->y, obs->nx, obs->ny, obs->w, obs->kappa, obs->id, obs->hs};
  a.lpts = PointTable{src->x, src->y, src->nx, src->ny, src->w, src->kappa, src->id, src->hs};
  a.tp_pt = reinterpret_cast<const int*>(d + o1);
  a.tp_s0 = reinterpret_cast<const int*>(d + o2);
  a.tp_s1 = reinterpret_cast<const int*>(d + o3);
  a.lp_pt = reinterpret_cast<const int*>(d + o4);
  a.lp_s0 = reinterpret_cast<const int*>(d + o5);
  a.lp_s1 = reinterpret_cast<const int*>(d + o6);
  a.jobs = reinterpret_cast<const TileJob*>(d + o7);
  a.chunks = reinterpret_cast<const TileChunk*>(d + o8);
  a.nchunks = (int)ch.size();
  a.out = reinterpret_cast<double2*>(out);
  a.status = reinterpret_cast<int*>(d + o9);
  a.kps = reinterpret_cast<const KernelParams*>(d + o10);
  CKE(launch_tiles(a, s));
  int st = 0;
  CKE(cudaMemcpyAsync(&st, a.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKE(cudaStreamSynchronize(s));
  return status_code(st);
}

int symhss_column_id(void* A, int m, int n, int lda, long long strideA, int batch, double tol, int fixed_rank,
                     int* rank, int* perm, void* T, long long strideT, void* stream) {
  if (batch < 0 || m < 0 || n < 0 || lda < m || lda < 1 || !(tol >= 0) || !std::isfinite(tol))
    return SYMHSS_ERR_INVALID;
  if (batch == 0) return SYMHSS_OK;
  if (!A || !rank || !perm || !T) return SYMHSS_ERR_INVALID;
  if (strideA < (long long)lda * n || strideT < (long long)(n / 2) * ((n + 1) / 2)) return SYMHSS_ERR_INVALID;
  const size_t smem = (size_t)m * 16 + (size_t)n * 16;  // the ID kernel's shared memory
  if (smem > 200 * 1024) return SYMHSS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<IdJob> jobs(batch);
  for (int b = 0; b < batch; ++b) {
    IdJob& j = jobs[b];
    j.m_off = strideA * b; j.m = m; j.n = n; j.ld = lda; j.start = 0; j.fixed = fixed_rank < 0 ? -1 : fixed_rank;
    j.t_off = strideT * b; j.perm_off = (long long)n * b; j.out_idx = b;
  }
  TmpBuf buf;
  const size_t bytes = jobs.size() * sizeof(IdJob) + batch * sizeof(double) + 64;
  CKE(buf.alloc(bytes));
  CKE(cudaMemcpyAsync(buf.p, jobs.data(), jobs.size() * sizeof(IdJob), cudaMemcpyHostToDevice, s));
  char* d = reinterpret_cast<char*>(buf.p);
  double* ref = reinterpret_cast<double*>(d + ((jobs.size() * sizeof(IdJob) + 15) & ~size_t(15)));
  int* status = reinterpret_cast<int*>(ref + batch);
  CKE(cudaMemsetAsync(status, 0, sizeof(int), s));
  IdLaunch a;
  a.mats = reinterpret_cast<double2*>(A);
  a.tbuf = reinterpret_cast<double2*>(T);
  a.perm = perm;
  a.rank = rank;
  a.ref = ref;
  a.jobs = reinterpret_cast<const IdJob*>(d);
  a.njobs = batch;
  a.tol = tol;
  a.status = status;
  a.max_m = m > 0 ? m : 1;
  a.max_n = n > 0 ? n : 1;
  CKE(launch_cpqr(a, s));
  int st = 0;
  CKE(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKE(cudaStreamSynchronize(s));
  return status_code(st);
}

int symhss_sketch(const void* A, int m, int n, int lda, long long strideA, int batch, int s_rows,
                  unsigned long long seed, void* Y, int ldy, long long strideY, void* stream) {
  if (batch < 0 || m < 0 || n < 0 || s_rows < 0 || lda < m || lda < 1 || ldy < s_rows || ldy < 1)
    return SYMHSS_ERR_INVALID;
  if (m > 65536 || s_rows > 1024) return SYMHSS_ERR_INVALID;
  if (batch == 0 || n == 0 || s_rows == 0) return SYMHSS_OK;
  if (!A || !Y || strideA < (long long)lda * n || strideY < (long long)ldy * n) return SYMHSS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const int mpad = sketch_mpad(m), n2pad = sketch_n2pad(n);
  const size_t sbytes = sketch_slice_bytes(mpad, n2pad);
  std::vector<SketchJob> jobs(batch);
  std::vector<SketchColWork> cw;
  std::vector<SketchTile> tiles;
  const int mtiles = (s_rows + 127) / 128;
  for (int b = 0; b < batch; ++b) {
    SketchJob& j = jobs[b];
    j.m_off = strideA * b; j.m = m; j.n = n; j.ld = lda; j.mpad = mpad; j.n2pad = n2pad; j.s = s_rows;
    j.y_off = strideY * b; j.ldy = ldy; j.slice_off = (long long)sbytes * b; j.exp_off = (long long)2 * n * b;
    j.stream_id = b;
    for (int c = 0; c < n; ++c) cw.push_back(SketchColWork{b, c});
    for (int cb = 0; cb < n2pad / 32; ++cb)
      for (int mt = 0; mt < mtiles; ++mt) tiles.push_back(SketchTile{b, cb, mt});
  }
  TmpBuf slices, meta;
  CKE(slices.alloc(sbytes * batch));
  const size_t o_exp = 0, o_jobs = ((size_t)2 * n * batch * sizeof(int) + 255) & ~size_t(255);
  const size_t o_cw = o_jobs + ((jobs.size() * sizeof(SketchJob) + 255) & ~size_t(255));
  const size_t o_tiles = o_cw + ((cw.size() * sizeof(SketchColWork) + 255) & ~size_t(255));
  const size_t o_status = o_tiles + ((tiles.size() * sizeof(SketchTile) + 255) & ~size_t(255));
  const size_t total = o_status + 256;
  CKE(meta.alloc(total));
  std::vector<char> host(total, 0);
  std::memcpy(host.data() + o_jobs, jobs.data(), jobs.size() * sizeof(SketchJob));
  std::memcpy(host.data() + o_cw, cw.data(), cw.size() * sizeof(SketchColWork));
  std::memcpy(host.data() + o_tiles, tiles.data(), tiles.size() * sizeof(SketchTile));
  CKE(cudaMemcpyAsync(meta.p, host.data(), total, cudaMemcpyHostToDevice, s));
  char* d = reinterpret_cast<char*>(meta.p);
  SketchLaunch a;
  a.mats = reinterpret_cast<const double2*>(A);
  a.slices = reinterpret_cast<uint8_t*>(slices.p);
  a.exps = reinterpret_cast<int*>(d + o_exp);
  a.y = reinterpret_cast<double2*>(Y);
  a.jobs = reinterpret_cast<const SketchJob*>(d + o_jobs);
  a.colwork = reinterpret_cast<const SketchColWork*>(d + o_cw);
  a.ncolwork = (int)cw.size();
  a.tiles = reinterpret_cast<const SketchTile*>(d + o_tiles);
  a.ntiles = (int)tiles.size();
  a.seed = seed;
  a.status = reinterpret_cast<int*>(d + o_status);
  CKE(launch_sketch(a, s));
  int st = 0;
  CKE(cudaMemcpyAsync(&st, a.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKE(cudaStreamSynchronize(s));
  if (st & ST_TIMEOUT) return SYMHSS_ERR_TIMEOUT;
  return status_code(st);
}

int symhss_lu_batched(void* A, int n, int lda, long long strideA, int batch, int* ipiv, int* info, void* stream) {
  if (batch < 0 || n < 0 || lda < n || lda < 1) return SYMHSS_ERR_INVALID;
  if (batch == 0 || n == 0) return SYMHSS_OK;
  if (!A || !ipiv || !info || strideA < (long long)lda * n) return SYMHSS_ERR_INVALID;
  if (2 * (size_t)n * 16 > 220 * 1024) return SYMHSS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<LuJob> jobs(batch);
  for (int b = 0; b < batch; ++b) {
    jobs[b].a_off = strideA * b; jobs[b].n = n; jobs[b].ld = lda; jobs[b].piv_off = (long long)n * b;
    jobs[b].info_idx = b;
  }
  TmpBuf buf;
  CKE(buf.alloc(jobs.size() * sizeof(LuJob) + 64));
  CKE(cudaMemcpyAsync(buf.p, jobs.data(), jobs.size() * sizeof(LuJob), cudaMemcpyHostToDevice, s));
  int* status = reinterpret_cast<int*>(reinterpret_cast<char*>(buf.p) + ((jobs.size() * sizeof(LuJob) + 15) & ~size_t(15)));
  CKE(cudaMemsetAsync(status, 0, sizeof(int), s));
  LuLaunch a;
  a.base = reinterpret_cast<double2*>(A);
  a.piv = ipiv;
  a.info = info;
  a.jobs = reinterpret_cast<const LuJob*>(buf.p);
  a.njobs = batch;
  a.max_n = n;
  a.status = status;
  TmpBuf zimg;  // tensor-core product scratch of the blocked LU
  a.zimg_bytes = zgemm_lu_img_bytes(batch, n);
  if (a.zimg_bytes > 0) {
    CKE(zimg.alloc((size_t)a.zimg_bytes));
    a.zimg = reinterpret_cast<unsigned char*>(zimg.p);
  }
  CKE(launch_getrf(a, s));
  int st = 0;
  CKE(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKE(cudaStreamSynchronize(s));
  if (st & ST_BAD_INDEX) return SYMHSS_ERR_DEVICE;
  if (st & ST_TIMEOUT) return SYMHSS_ERR_TIMEOUT;
  return SYMHSS_OK;  // singular blocks are reported in info
}

int symhss_lu_solve_batched(const void* LU, int n, int lda, long long strideA, const int* ipiv, void* B, int nrhs,
                            int ldb, long long strideB, int batch, void* stream) {
  if (batch < 0 || n < 0 || nrhs < 0 || lda < n || ldb < n || lda < 1 || ldb < 1) return SYMHSS_ERR_INVALID;
  if (batch == 0 || n == 0 || nrhs == 0) return SYMHSS_OK;
  if (!LU || !ipiv || !B || strideA < (long long)lda * n || strideB < (long long)ldb * nrhs)
    return SYMHSS_ERR_INVALID;
  if ((size_t)n * 4 + 16 + (size_t)4 * n * 16 > 220 * 1024) return SYMHSS_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<RsJob> jobs(batch);
  for (int b = 0; b < batch; ++b) {
    jobs[b].a_off = strideA * b; jobs[b].n = n; jobs[b].lda = lda; jobs[b].piv_off = (long long)n * b;
    jobs[b].b_off = strideB * b; jobs[b].ldb = ldb; jobs[b].nrhs = nrhs;
  }
  TmpBuf buf;
  const size_t o_status = (jobs.size() * sizeof(RsJob) + 15) & ~size_t(15);
  CKE(buf.alloc(o_status + 16));
  CKE(cudaMemcpyAsync(buf.p, jobs.data(), jobs.size() * sizeof(RsJob), cudaMemcpyHostToDevice, s));
  int* status = reinterpret_cast<int*>(reinterpret_cast<char*>(buf.p) + o_status);
  CKE(cudaMemsetAsync(status, 0, sizeof(int), s));
  RsLaunch a;
  a.abase = reinterpret_cast<const double2*>(LU);
  a.piv = ipiv;
  a.bbase = reinterpret_cast<double2*>(B);
  a.jobs = reinterpret_cast<const RsJob*>(buf.p);
  a.njobs = batch;
  a.max_rhs = nrhs;
  a.max_n = n;
  a.status = status;
  TmpBuf zimg;  // tensor-core product scratch of the blocked solve
  a.zimg_bytes = zgemm_rs_img_bytes(batch, n, nrhs);
  if (a.zimg_bytes > 0) {
    CKE(zimg.alloc((size_t)a.zimg_bytes));
    a.zimg = reinterpret_cast<unsigned char*>(zimg.p);
  }
  // inverses of the diagonal blocks for batches of fewer than 32 matrices; larger batches keep
  // the substitutions with the right-hand sides on the lanes (both paths reachable from here)
  TmpBuf dinv;
  if (batch < 32 && nrhs > 4) {
    a.dinv_bytes = getrs_dinv_bytes(batch, n);
    CKE(dinv.alloc((size_t)a.dinv_bytes));
    a.dinv = reinterpret_cast<double2*>(dinv.p);
  }
  CKE(launch_getrs(a, s));
  int st = 0;
  CKE(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKE(cudaStreamSynchronize(s));
  return status_code(st);
}

}  // extern "C"
