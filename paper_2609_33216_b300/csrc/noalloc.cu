// Column ID entry point that performs no device memory allocation.
//
// symhss_column_id allocates a small device buffer on every call (job
// descriptors, per-matrix reference norms and a status word).  Some callers
// cannot do that: code running under a fixed device-memory budget or inside an
// allocator they do not own, and latency-critical loops where the implicit
// device-wide synchronisation of cudaMalloc / cudaFree is not acceptable.  This
// variant keeps that scratch in one file-scope __device__ array instead, of
// fixed size kMaxBatch jobs, which every GPU that loads the library holds until
// the process exits.
//
// The host never dereferences the array's symbol: on the first call made on a
// device it asks the runtime for the array's device address (with that device
// current) and caches it; later calls on the same device reuse the cached
// address.  Because that first call talks to the runtime, it should be made
// before any stream capture begins.  The cached address belongs to the device's
// current context: a cudaDeviceReset while the library is in use would leave it
// stale, so devices the library has used must not be reset.  All calls share the one array, and each
// call leaves its job descriptors and status word behind: the status word is
// cleared at the start of every call, and calls whose work overlaps on the GPU
// (different streams or host threads without ordering between them) race on the
// array and must not be issued.
#include <cmath>
#include <mutex>

#include "common.cuh"

using namespace symhss;

namespace {

constexpr int kMaxBatch = 4096;
constexpr size_t kJobsBytes = ((size_t)kMaxBatch * sizeof(IdJob) + 255) & ~size_t(255);
constexpr size_t kRefBytes = ((size_t)kMaxBatch * sizeof(double) + 255) & ~size_t(255);
constexpr size_t kScratchBytes = kJobsBytes + kRefBytes + 256;

static __device__ __align__(256) unsigned char g_id_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of the scratch array for the current device (set up once per device).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_id_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = reinterpret_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Uniform-batch job descriptors and a cleared status word, written on the device.
__global__ void fill_id_jobs(IdJob* jobs, int* status, int batch, int m, int n, int lda, long long stride_a,
                             int fixed, long long stride_t) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) *status = 0;
  if (b >= batch) return;
  IdJob j;
  j.m_off = stride_a * b;
  j.m = m;
  j.n = n;
  j.ld = lda;
  j.start = 0;
  j.fixed = fixed;
  j.t_off = stride_t * b;
  j.perm_off = (long long)n * b;
  j.out_idx = b;
  jobs[b] = j;
}

int to_status(cudaError_t e) { return e == cudaErrorMemoryAllocation ? SYMHSS_ERR_NOMEM : SYMHSS_ERR_CUDA; }

}  // namespace

extern "C" int symhss_column_id_noalloc(void* A, int m, int n, int lda, long long strideA, int batch, double tol,
                                        int fixed_rank, int* rank, int* perm, void* T, long long strideT,
                                        void* stream) {
  if (batch < 0 || m < 0 || n < 0 || lda < m || lda < 1 || !(tol >= 0) || !std::isfinite(tol))
    return SYMHSS_ERR_INVALID;
  if (batch > kMaxBatch) return SYMHSS_ERR_INVALID;
  if (batch == 0) return SYMHSS_OK;
  if (!A || !rank || !perm || !T) return SYMHSS_ERR_INVALID;
  if (strideA < (long long)lda * n || strideT < (long long)(n / 2) * ((n + 1) / 2)) return SYMHSS_ERR_INVALID;
  if ((size_t)m * 16 + (size_t)n * 16 > 200 * 1024) return SYMHSS_ERR_INVALID;  // ID kernel shared memory
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return to_status(e);
  IdJob* jobs = reinterpret_cast<IdJob*>(base);
  double* ref = reinterpret_cast<double*>(base + kJobsBytes);
  int* status = reinterpret_cast<int*>(base + kJobsBytes + kRefBytes);
  fill_id_jobs<<<(batch + 127) / 128, 128, 0, s>>>(jobs, status, batch, m, n, lda, strideA,
                                                   fixed_rank < 0 ? -1 : fixed_rank, strideT);
  e = cudaGetLastError();
  if (e != cudaSuccess) return to_status(e);
  IdLaunch a;
  a.mats = reinterpret_cast<double2*>(A);
  a.tbuf = reinterpret_cast<double2*>(T);
  a.perm = perm;
  a.rank = rank;
  a.ref = ref;
  a.jobs = jobs;
  a.njobs = batch;
  a.tol = tol;
  a.status = status;
  a.max_m = m > 0 ? m : 1;
  a.max_n = n > 0 ? n : 1;
  e = launch_cpqr(a, s);
  if (e != cudaSuccess) return to_status(e);
  int st = 0;
  e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return to_status(e);
  return st ? SYMHSS_ERR_DEVICE : SYMHSS_OK;
}
