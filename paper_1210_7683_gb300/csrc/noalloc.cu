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
// GPU (for example on two streams) race on it; the status words (the heritability
// check and the counter of singular pairs) are cleared at the start of each call.
//
// The array's device address is looked up on every call, with the caller's current
// device: a host application that tears its CUDA context down and creates a new one
// (cudaDeviceReset) gets the array of the new context's module, never a stale address.
#include <cfloat>
#include <cstring>

#include "gwas_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// status[0] bits: 1 = some h2 outside [0, 1] (or NaN); 2 = some D_j = h2 lambda + 1 - h2 has an
// entry <= 1e-12 of its largest (M_j not positive definite, the condition gwas_setup checks).
__global__ void __launch_bounds__(256) check_h2_kernel(const double* __restrict__ h2, const double* __restrict__ lam,
                                                       int n, unsigned long long* status) {
  const int j = blockIdx.x;
  const double h = h2[j];
  if (!(h >= 0.0 && h <= 1.0)) {
    if (threadIdx.x == 0) atomicOr(status, 1ull);
    return;
  }
  double lo = DBL_MAX, hi = -DBL_MAX;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double d = h * lam[k] + (1.0 - h);
    lo = fmin(lo, d);
    hi = fmax(hi, d);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  __shared__ double slo[8], shi[8];
  if ((threadIdx.x & 31) == 0) {
    slo[threadIdx.x / 32] = lo;
    shi[threadIdx.x / 32] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x / 32); ++w) {
      lo = fmin(lo, slo[w]);
      hi = fmax(hi, shi[w]);
    }
    if (!(lo > 1e-12 * hi)) atomicOr(status, 2ull);
  }
}

// True when p is device (or managed) memory that kernels on `dev` may read and write.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

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
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  // every array must be device memory of the current device: kernels read and write them directly
  if (!on_device(lam, dev) || !on_device(Yt, dev) || !on_device(h2, dev) || !on_device(out, dev) ||
      (m > 0 && !on_device(Xt, dev)) || (pm1 > 0 && !on_device(XLt, dev)))
    return GWAS_ERR_ARG;
  void* p0 = nullptr;
  if (cudaGetSymbolAddress(&p0, g_noalloc_scratch) != cudaSuccess || !p0) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  unsigned char* base = (unsigned char*)p0;
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
  c.d_status = (unsigned long long*)base;  // [0] heritability check, [1] singular-pair counter
  double* R = (double*)(base + 256);
  double* consts = (double*)(base + 256 + ((r_bytes + 255) & ~size_t(255)));
  if (cudaMemsetAsync(base, 0, 16, c.stream) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  // the heritabilities first: h2 outside [0, 1] or a non-positive D_j stops the call before any
  // result is written
  check_h2_kernel<<<t, 256, 0, c.stream>>>(h2, lam, n, c.d_status);
  unsigned long long st[2] = {0, 0};
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(st, base, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
      cudaStreamSynchronize(c.stream) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  if (st[0] & 1ull) return GWAS_ERR_ARG;
  if (st[0] & 2ull) return GWAS_ERR_NOT_SPD;
  if (m > 0) {
    launch_prep_fp64(&c, Yt, t, h2, R, consts);
    if (output == GWAS_OUT_FULL_B) {
      launch_fused_fp64(&c, 0, m, 0, t, m, R, consts, out);
    } else {
      void* pair[2] = {out, (float*)out + (size_t)t * m};
      launch_fused_fp64(&c, 0, m, 0, t, m, R, consts, pair);
    }
  }
  if (cudaGetLastError() != cudaSuccess) return GWAS_ERR_CUDA;
  if (cudaMemcpyAsync(st, base, sizeof st, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
      cudaStreamSynchronize(c.stream) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  if (singular) *singular = (int64_t)st[1];
  return st[1] ? GWAS_ERR_SINGULAR_PAIRS : GWAS_OK;
}
