// Self-tests.  The bounded waits that every kernel of the library uses: a wait on an
// mbarrier that nothing completes must give up after its limit, record the failure in
// the status word and return, leaving the CUDA context usable.  No fault, trap or
// endless loop is involved.  And the epilogue's reciprocal and square root beside CUDA's
// correctly rounded ones.
#include <chrono>

#include "gwas_internal.cuh"
#include "tc.cuh"

namespace {

__global__ void stuck_wait_kernel(unsigned long long* status, uint64_t limit_ns, unsigned long long* waited_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);  // one arrival expected; none will come
    abort = 0;
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t t0 = tc::globaltimer_ns();
    tc::mbar_wait_limit(&bar, 0, status, &abort, limit_ns);
    *waited_ns = tc::globaltimer_ns() - t0;
  }
}

__global__ void epilogue_math_kernel(const float* __restrict__ x, int count, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float v = x[i];
  out[4 * i + 0] = tc::rcp_nr(v);
  out[4 * i + 1] = __frcp_rn(v);
  out[4 * i + 2] = tc::sqrt_approx(v);
  out[4 * i + 3] = __fsqrt_rn(v);
}

}  // namespace

extern "C" int gwas_check_epilogue_math(int device, const float* x, int count, float* out) {
  if (!x || !out || count < 1 || count > (1 << 20)) return GWAS_ERR_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_ARG;
  }
  float* d = nullptr;
  if (cudaMalloc(&d, sizeof(float) * 5 * (size_t)count) != cudaSuccess) {
    cudaGetLastError();
    cudaSetDevice(prev);
    return GWAS_ERR_OOM;
  }
  int rc = GWAS_OK;
  if (cudaMemcpy(d, x, sizeof(float) * count, cudaMemcpyHostToDevice) != cudaSuccess) rc = GWAS_ERR_CUDA;
  if (rc == GWAS_OK) {
    epilogue_math_kernel<<<(count + 255) / 256, 256>>>(d, count, d + count);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(out, d + count, sizeof(float) * 4 * (size_t)count, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = GWAS_ERR_CUDA;
  }
  if (rc) cudaGetLastError();
  cudaFree(d);
  cudaSetDevice(prev);
  return rc;
}

extern "C" int gwas_check_bounded_wait(int device, double limit_s, double* waited_s) {
  if (!(limit_s > 0) || limit_s > 10) return GWAS_ERR_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_ARG;
  }
  unsigned long long* d = nullptr;
  int rc = GWAS_OK;
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    cudaSetDevice(prev);
    return GWAS_ERR_OOM;
  }
  cudaMemset(d, 0, 2 * sizeof(unsigned long long));
  stuck_wait_kernel<<<1, 32>>>(d, (uint64_t)(limit_s * 1e9), d + 1);
  unsigned long long h[2] = {0, 0};
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    rc = GWAS_ERR_CUDA;
  } else {
    rc = h[0] ? GWAS_ERR_TIMEOUT : GWAS_OK;
    if (waited_s) *waited_s = (double)h[1] * 1e-9;
  }
  cudaFree(d);
  cudaSetDevice(prev);
  return rc;
}
