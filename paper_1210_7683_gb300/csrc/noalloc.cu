// Allocation-free entry point: the FP64 per-trait preparation and the fused FP64
// contraction + solve, with their scratch in a fixed file-scope device array
// instead of memory from cudaMalloc.
//
// Some callers cannot allocate device memory: code that runs inside a host
// application whose memory manager owns the whole device (a framework's caching
// allocator, a fixed arena set aside at start-up), or plug-in code that is only
// handed buffers and a stream.  They pass already-rotated inputs and the output
// buffers; this entry point uses nothing else on the device.
//
// Limits and sharing: the scratch holds at most kScratchBytes (8 MiB); every GPU
// that loads the library keeps this array until the process exits.  All calls
// share it and it keeps the last call's contents, so two calls that overlap on the
// GPU (for example on two streams) race on it; the counter of singular pairs is
// cleared at the start of each call.
#include <cstring>

#include "gwas_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once with that device current.
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" int gwas_solve_fp64_noalloc(int n, int pm1, const double* lam, const double* XLt, const double* Xt,
                                       int64_t m, const double* Yt, const double* h2, int t, int output, void* out,
                                       void* stream, int64_t* singular) {
  if (singular) *singular = 0;
  if (n < 1 || pm1 < 0 || pm1 > GWAS_MAX_PM1 || n <= pm1 + 1 || t < 1 || m < 0) return GWAS_ERR_ARG;
  if (!lam || !Yt || !h2 || !out || (m > 0 && !Xt) || (pm1 > 0 && !XLt)) return GWAS_ERR_ARG;
  if (output != GWAS_OUT_FULL_B && output != GWAS_OUT_LAST_SE) return GWAS_ERR_ARG;
  const int p = pm1 + 1;
  const size_t r_bytes = sizeof(double) * (size_t)t * (p + 1) * n;
  const size_t c_bytes = sizeof(double) * (size_t)t * consts_stride(pm1);
  const size_t need = 256 + ((r_bytes + 255) & ~size_t(255)) + c_bytes;
  if (need > kScratchBytes) return GWAS_ERR_UNSUPPORTED;  // t (p+1) n + t (p^2 - p + 1) doubles exceed 8 MiB
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  if (!g_scratch_addr[dev]) {
    void* p0 = nullptr;
    if (cudaGetSymbolAddress(&p0, g_noalloc_scratch) != cudaSuccess || !p0) {
      cudaGetLastError();
      return GWAS_ERR_CUDA;
    }
    g_scratch_addr[dev] = p0;
  }
  unsigned char* base = (unsigned char*)g_scratch_addr[dev];
  // a context object on the host stack carries the launch parameters; it owns no device memory
  gwas_ctx c;
  c.n = n;
  c.pm1 = pm1;
  c.p = p;
  c.t = t;
  c.device = dev;
  c.precision = GWAS_FP64;
  c.output = output;
  c.stream = (cudaStream_t)stream;
  c.lam = const_cast<double*>(lam);
  c.XLt = const_cast<double*>(XLt);
  c.Xt = const_cast<double*>(Xt);
  c.d_status = (unsigned long long*)base;  // [0] unused, [1] singular-pair counter
  double* R = (double*)(base + 256);
  double* consts = (double*)(base + 256 + ((r_bytes + 255) & ~size_t(255)));
  if (cudaMemsetAsync(base, 0, 16, c.stream) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  if (m > 0) {
    launch_prep_fp64(&c, Yt, t, h2, R, consts);
    if (output == GWAS_OUT_FULL_B) {
      launch_fused_fp64(&c, 0, m, 0, t, m, R, consts, out);
    } else {
      void* pair[2] = {out, (float*)out + (size_t)t * m};
      launch_fused_fp64(&c, 0, m, 0, t, m, R, consts, pair);
    }
  }
  unsigned long long cnt = 0;
  if (cudaGetLastError() != cudaSuccess) return GWAS_ERR_CUDA;
  if (cudaMemcpyAsync(&cnt, base + 8, sizeof cnt, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
      cudaStreamSynchronize(c.stream) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  if (singular) *singular = (int64_t)cnt;
  return cnt ? GWAS_ERR_SINGULAR_PAIRS : GWAS_OK;
}
