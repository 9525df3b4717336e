// C interface of the GWAS library: contexts, device memory, argument checks and the
// orchestration of the preloop and loop phases of Algorithm 5 (Section 3).
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "fused.cuh"
#include "gwas_internal.cuh"

static thread_local std::string g_setup_err;

namespace {

// One cuSOLVER handle per device for the whole process, created on first use: creating a
// handle and its first eigensolver call cost several milliseconds that every gwas_setup
// would otherwise pay.  The mutex serialises contexts of different host threads that run
// their eigendecompositions at the same time (a handle is bound to one stream at a time).
struct SolverCache {
  std::mutex mu;
  std::map<int, cusolverDnHandle_t> handles;
};
SolverCache& solver_cache() {
  static SolverCache* s = new SolverCache;  // never destroyed: handles outlive every context
  return *s;
}

// Device memory of every context comes from one stream-ordered pool per device that keeps what
// contexts give back (its release threshold is unlimited): a context set up after another reuses
// that memory instead of mapping it again.  Mapping and unmapping are not free: a step of the
// n = 1000, m = 10^6, t = 10^4 workload allocates ~10 GB, which cudaMalloc maps in ~1 ms and
// cudaFree unmaps in ~5 ms.  gwas_pool_trim gives kept memory back.  Allocations and frees run on
// the pool's own stream and are waited for, so a buffer is usable from every stream on return,
// and the pool never hands out memory whose free is still pending (internal dependencies off).
// GWAS_POOL=0 in the environment (read once) uses cudaMalloc/cudaFree instead.
struct DevicePool {
  cudaMemPool_t pool = nullptr;
  cudaStream_t stream = nullptr;
};
struct PoolCache {
  std::mutex mu;
  std::map<int, DevicePool> pools;
  int enabled = -1;
};
PoolCache& pool_cache() {
  static PoolCache* p = new PoolCache;  // never destroyed: pools outlive every context
  return *p;
}

// The pool of `dev`, created on first use (`create`); null when pooling is off, the device has
// no memory pools, or it does not exist yet and `create` is false.
DevicePool device_pool(int dev, bool create = true) {
  PoolCache& pc = pool_cache();
  std::lock_guard<std::mutex> lk(pc.mu);
  if (pc.enabled < 0) {
    const char* e = std::getenv("GWAS_POOL");
    pc.enabled = (e && std::strcmp(e, "0") == 0) ? 0 : 1;
  }
  if (!pc.enabled) return {};
  auto it = pc.pools.find(dev);
  if (it != pc.pools.end()) return it->second;
  if (!create) return {};
  DeviceGuard guard(dev);
  DevicePool dp;
  int supported = 0;
  if (cudaDeviceGetAttribute(&supported, cudaDevAttrMemoryPoolsSupported, dev) != cudaSuccess || !supported) {
    cudaGetLastError();
    pc.pools[dev] = dp;
    return dp;
  }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  if (cudaMemPoolCreate(&dp.pool, &props) != cudaSuccess) {
    cudaGetLastError();
    pc.pools[dev] = DevicePool{};
    return {};
  }
  uint64_t keep = ~uint64_t(0);
  int off = 0;
  if (cudaMemPoolSetAttribute(dp.pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
      cudaMemPoolSetAttribute(dp.pool, cudaMemPoolReuseAllowInternalDependencies, &off) != cudaSuccess ||
      cudaStreamCreateWithFlags(&dp.stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cudaMemPoolDestroy(dp.pool);
    pc.pools[dev] = DevicePool{};
    return {};
  }
  pc.pools[dev] = dp;
  return dp;
}

// Device memory from the pool (or cudaMalloc), aligned to 256 bytes.
cudaError_t dev_malloc(int dev, void** p, size_t bytes) {
  DevicePool dp = device_pool(dev);
  if (!dp.pool) return cudaMalloc(p, bytes);
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, dp.pool, dp.stream);
  if (e == cudaErrorMemoryAllocation) {
    // the pool's free blocks may hold the room in pieces too small for this buffer: give them
    // back to the device and try once more
    cudaGetLastError();
    cudaMemPoolTrimTo(dp.pool, 0);
    e = cudaMallocFromPoolAsync(p, bytes, dp.pool, dp.stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(dp.stream);
  if (e == cudaSuccess && (reinterpret_cast<uintptr_t>(*p) & 255)) {
    cudaFreeAsync(*p, dp.stream);
    cudaStreamSynchronize(dp.stream);
    *p = nullptr;
    return cudaMalloc(p, bytes);  // not expected: pool blocks are at least 512-byte aligned
  }
  if (e != cudaSuccess) *p = nullptr;
  return e;
}

// Gives memory back. Like cudaFree it first waits for all work on the device, so no kernel or
// copy still uses the buffer when the pool may hand it out again.
void dev_free(int dev, void* p, bool pooled) {
  if (!p) return;
  if (!pooled) {
    cudaFree(p);
    return;
  }
  DevicePool dp = device_pool(dev);
  DeviceGuard guard(dev);
  cudaDeviceSynchronize();
  cudaFreeAsync(p, dp.stream);
  cudaStreamSynchronize(dp.stream);
}

std::string fmt(const char* f, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, f);
  vsnprintf(buf, sizeof buf, f, ap);
  va_end(ap);
  return buf;
}

}  // namespace

int ctx_fail(gwas_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg; else g_setup_err = msg;
  return code;
}

bool ctx_cuda_ok(gwas_ctx* c, cudaError_t e, const char* what, int* rc) {
  if (e == cudaSuccess) return true;
  cudaGetLastError();
  *rc = ctx_fail(c, e == cudaErrorMemoryAllocation ? GWAS_ERR_OOM : GWAS_ERR_CUDA,
                 fmt("%s: %s", what, cudaGetErrorString(e)));
  return false;
}

int ctx_alloc(gwas_ctx* c, size_t bytes, void** out) {
  *out = nullptr;
  size_t b = (bytes + 255) & ~size_t(255);
  if (b == 0) b = 256;
  if (c->budget && c->allocated + b > c->budget)
    return ctx_fail(c, GWAS_ERR_OOM, fmt("allocation of %zu bytes exceeds the HBM budget (%zu of %zu in use)", b,
                                         c->allocated, c->budget));
  void* p = nullptr;
  const bool pooled = device_pool(c->device).pool != nullptr;
  cudaError_t e = dev_malloc(c->device, &p, b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, GWAS_ERR_OOM, fmt("device allocation of %zu bytes: %s", b, cudaGetErrorString(e)));
  }
  c->bufs.push_back({p, b, pooled});
  c->allocated += b;
  *out = p;
  return GWAS_OK;
}

void ctx_free(gwas_ctx* c, void* p) {
  if (!p) return;
  for (size_t i = 0; i < c->bufs.size(); ++i)
    if (c->bufs[i].ptr == p) {
      dev_free(c->device, p, c->bufs[i].pooled);
      c->allocated -= c->bufs[i].bytes;
      c->bufs.erase(c->bufs.begin() + i);
      return;
    }
}

int ptr_kind(gwas_ctx* c, const void* p, bool* is_device) {
  cudaPointerAttributes a;
  *is_device = false;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_OK;  // unregistered host memory
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
    if (a.type == cudaMemoryTypeDevice && a.device != c->device)
      return ctx_fail(c, GWAS_ERR_ARG, fmt("device pointer on device %d, context on device %d", a.device, c->device));
    *is_device = true;
  }
  return GWAS_OK;
}

// Whether the kernels can store a host output [p, p + bytes) directly: the device reads the
// CPU's page tables (Grace-class systems, where every address of the process is reachable
// from the device), both ends of the range are page-locked host memory mapped for the device,
// and the device addresses of the ends are as far apart as the host ones.  Page-locked memory
// is resident, so the stores never wait for a page fault.  GWAS_HOST_OUTPUT=staged in the
// environment keeps the staged copies.
static bool direct_host_output(gwas_ctx* c, void* p, size_t bytes, void** dptr, bool input = false) {
  if (bytes == 0) return false;
  if (const char* e = getenv("GWAS_HOST_OUTPUT"))
    if (!input && !strcmp(e, "staged")) return false;
  int ats = 0;
  if (cudaDeviceGetAttribute(&ats, cudaDevAttrPageableMemoryAccessUsesHostPageTables, c->device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (!ats) return false;
  cudaPointerAttributes a0, a1;
  const char* last = (const char*)p + bytes - 1;
  if (cudaPointerGetAttributes(&a0, p) != cudaSuccess || cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
    return false;
  if ((const char*)a1.devicePointer - (const char*)a0.devicePointer != (ptrdiff_t)(bytes - 1)) return false;
  *dptr = a0.devicePointer;
  return true;
}

// Whether a kernel can read the host input [p, p + bytes) directly, under the same conditions as
// direct_host_output (a device that reads the CPU's page tables, page-locked memory mapped for the
// device).  On this kind of system the copy engines' host -> device rate from page-locked buffers
// that have existed for a while fell to 17-54 GB/s in processes that followed other large GPU
// processes, while kernel accesses to the same memory kept the link's rate.
// GWAS_HOST_INPUT=staged in the environment keeps the copies.
static bool direct_host_input(gwas_ctx* c, const void* p, size_t bytes, const void** dptr) {
  if (const char* e = getenv("GWAS_HOST_INPUT"))
    if (!strcmp(e, "staged")) return false;
  void* d = nullptr;
  if (!direct_host_output(c, const_cast<void*>(p), bytes, &d, true)) return false;
  *dptr = d;
  return true;
}

int ctx_upload(gwas_ctx* c, const void* src, size_t bytes, void* dst) {
  bool dev;
  int rc = ptr_kind(c, src, &dev);
  if (rc) return rc;
  if (!ctx_cuda_ok(c, cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
                   "upload", &rc))
    return rc;
  return GWAS_OK;
}

static cudaEvent_t pool_event(gwas_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(gwas_ctx* ctx, const char* name) : c(ctx), idx(SIZE_MAX) {
  if (!c->profile) return;
  ProfPending p{name, pool_event(c), pool_event(c)};
  cudaEventRecord(p.start, c->stream);
  idx = c->pending.size();
  c->pending.push_back(p);
}

ProfScope::~ProfScope() {
  if (idx != SIZE_MAX) cudaEventRecord(c->pending[idx].stop, c->stream);
}

void prof_flush(gwas_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
      auto& e = c->prof[p.name];
      e.first += ms;
      e.second += 1;
    } else {
      cudaGetLastError();
    }
    c->event_pool.push_back(p.start);
    c->event_pool.push_back(p.stop);
  }
  c->pending.clear();
}

extern "C" int gwas_kernel_time(const gwas_ctx* c, const char* kernel, double* ms, int64_t* launches) {
  if (!c || !kernel) return GWAS_ERR_ARG;
  auto it = c->prof.find(kernel);
  if (ms) *ms = it == c->prof.end() ? 0.0 : it->second.first;
  if (launches) *launches = it == c->prof.end() ? 0 : it->second.second;
  return GWAS_OK;
}

extern "C" void gwas_reset_timers(gwas_ctx* c) {
  if (c) c->prof.clear();
}

extern "C" void gwas_default_opts(gwas_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->precision = GWAS_MIXED;
  o->output = GWAS_OUT_LAST_SE;
}

static void destroy_impl(gwas_ctx* c) {
  if (!c) return;
  int dev;
  bool have = cudaGetDevice(&dev) == cudaSuccess;
  cudaSetDevice(c->device);
  serve_shutdown(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  prof_flush(c);
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  c->event_pool.clear();
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  for (int k = 0; k < 2; ++k) {
    if (c->ev_compute[k]) cudaEventDestroy(c->ev_compute[k]);
    if (c->ev_copy[k]) cudaEventDestroy(c->ev_copy[k]);
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  mixed_free(c);
  mixed_destroy(c);
  if (!c->bufs.empty()) cudaDeviceSynchronize();
  for (auto& b : c->bufs) {
    if (!b.pooled) {
      cudaFree(b.ptr);
      continue;
    }
    cudaFreeAsync(b.ptr, device_pool(c->device).stream);
  }
  if (!c->bufs.empty() && device_pool(c->device).stream) cudaStreamSynchronize(device_pool(c->device).stream);
  c->bufs.clear();
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  if (have) cudaSetDevice(dev);
  delete c;
}

extern "C" void gwas_destroy(gwas_ctx* c) { destroy_impl(c); }

static int pool_device_ok(int device) {
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  return (device < 0 || device >= count) ? GWAS_ERR_ARG : GWAS_OK;
}

extern "C" int gwas_pool_info(int device, uint64_t* reserved, uint64_t* used) {
  if (reserved) *reserved = 0;
  if (used) *used = 0;
  if (int rc = pool_device_ok(device)) return rc;
  DevicePool dp = device_pool(device, false);
  if (!dp.pool) return GWAS_OK;
  uint64_t r = 0, u = 0;
  if (cudaMemPoolGetAttribute(dp.pool, cudaMemPoolAttrReservedMemCurrent, &r) != cudaSuccess ||
      cudaMemPoolGetAttribute(dp.pool, cudaMemPoolAttrUsedMemCurrent, &u) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  if (reserved) *reserved = r;
  if (used) *used = u;
  return GWAS_OK;
}

extern "C" int gwas_pool_trim(int device, uint64_t keep_bytes) {
  if (int rc = pool_device_ok(device)) return rc;
  DevicePool dp = device_pool(device, false);
  if (!dp.pool) return GWAS_OK;
  if (cudaMemPoolTrimTo(dp.pool, (size_t)keep_bytes) != cudaSuccess) {
    cudaGetLastError();
    return GWAS_ERR_CUDA;
  }
  return GWAS_OK;
}

extern "C" const char* gwas_last_error(const gwas_ctx* c) { return c ? c->err.c_str() : g_setup_err.c_str(); }

extern "C" int64_t gwas_singular_count(const gwas_ctx* c) { return c ? c->singular : 0; }

extern "C" int gwas_eig_info(const gwas_ctx* c, int* steps) {
  if (!c || !steps) return GWAS_ERR_ARG;
  *steps = c->eig_steps;
  return GWAS_OK;
}

extern "C" int gwas_fp4_info(gwas_ctx* c, int* ready, int64_t* launches) {
  if (!c) return GWAS_ERR_ARG;
  if (ready) *ready = c->precision == GWAS_MIXED ? mixed_fp4_ready(c) : 0;
  if (launches) *launches = c->fp4_launches;
  return GWAS_OK;
}

extern "C" int64_t gwas_kernel_launches(const gwas_ctx* c) { return c ? c->launches : 0; }

static int check_h2(gwas_ctx* c, const std::vector<double>& h2) {
  double lmin = c->h_lam.front(), lmax = c->h_lam.back();
  for (size_t j = 0; j < h2.size(); ++j) {
    double h = h2[j];
    if (!(h >= 0.0 && h <= 1.0)) return ctx_fail(c, GWAS_ERR_ARG, fmt("h2[%zu] = %g outside [0, 1]", j, h));
    double dmin = std::min(h * lmin + 1.0 - h, h * lmax + 1.0 - h);
    double dmax = std::max(h * lmin + 1.0 - h, h * lmax + 1.0 - h);
    if (!(dmin > 1e-12 * dmax))
      return ctx_fail(c, GWAS_ERR_NOT_SPD,
                      fmt("M_j not positive definite for trait %zu: min_k h2*lambda_k + 1 - h2 = %g", j, dmin));
  }
  return GWAS_OK;
}

extern "C" int gwas_setup(gwas_ctx** out, int n, int pm1, const double* phi, const double* XL, int t,
                          const double* h2, const gwas_opts* opts) {
  if (!out) return ctx_fail(nullptr, GWAS_ERR_ARG, "ctx pointer is NULL");
  *out = nullptr;
  gwas_opts o;
  gwas_default_opts(&o);
  if (opts) o = *opts;
  if (n < 1 || n > 16384) return ctx_fail(nullptr, GWAS_ERR_ARG, fmt("n = %d outside [1, 16384]", n));
  if (pm1 < 0 || pm1 > GWAS_MAX_PM1) return ctx_fail(nullptr, GWAS_ERR_UNSUPPORTED, fmt("p-1 = %d outside [0, 19]", pm1));
  if (n <= pm1 + 1) return ctx_fail(nullptr, GWAS_ERR_ARG, "need n > p");
  if (t < 1) return ctx_fail(nullptr, GWAS_ERR_ARG, "t must be >= 1");
  if (!phi || !h2 || (pm1 > 0 && !XL)) return ctx_fail(nullptr, GWAS_ERR_ARG, "NULL input array");
  if (o.precision != GWAS_FP64 && o.precision != GWAS_MIXED) return ctx_fail(nullptr, GWAS_ERR_ARG, "bad precision mode");
  if (o.output != GWAS_OUT_FULL_B && o.output != GWAS_OUT_LAST_SE) return ctx_fail(nullptr, GWAS_ERR_ARG, "bad output mode");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return ctx_fail(nullptr, GWAS_ERR_CUDA, "no CUDA device");
  }
  if (o.device < 0 || o.device >= ndev) return ctx_fail(nullptr, GWAS_ERR_ARG, "bad device ordinal");
  DeviceGuard guard(o.device);

  gwas_ctx* c = new gwas_ctx;
  c->n = n; c->pm1 = pm1; c->p = pm1 + 1; c->t = t; c->device = o.device;
  c->precision = o.precision; c->output = o.output; c->trait_block = o.trait_block; c->budget = o.hbm_budget;
  c->profile = o.profile != 0;
  if (o.tune_cache) {
    c->tune_cache = o.tune_cache;
    tune_apply_cache(c);
  }
  int rc = GWAS_OK;
  auto fail = [&](int code) { g_setup_err = c->err; destroy_impl(c); return code; };
  if (o.stream) {
    c->stream = (cudaStream_t)o.stream;
  } else {
    if (!ctx_cuda_ok(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream", &rc)) return fail(rc);
    c->own_stream = true;
  }
  if ((rc = ctx_alloc(c, 32, (void**)&c->d_status))) return fail(rc);
  cudaMemsetAsync(c->d_status, 0, 32, c->stream);

  // ---- eigendecomposition Phi = Z Lambda Z^T (Algorithm 5, eigendec), to FP64 accuracy: the
  // FP32 solver refined on the tensor cores (eig.cu), or the FP64 solver where that does not
  // converge (or under GWAS_EIG=fp64)
  if ((rc = ctx_alloc(c, sizeof(double) * n * n, (void**)&c->Z))) return fail(rc);
  if ((rc = ctx_alloc(c, sizeof(double) * n, (void**)&c->lam))) return fail(rc);
  double* phi_d = nullptr;
  if ((rc = ctx_alloc(c, sizeof(double) * n * n, (void**)&phi_d))) return fail(rc);
  if ((rc = ctx_upload(c, phi, sizeof(double) * n * n, phi_d))) return fail(rc);
  SolverCache& sc = solver_cache();
  std::unique_lock<std::mutex> solver_lock(sc.mu);
  cusolverDnHandle_t h = sc.handles.count(c->device) ? sc.handles[c->device] : nullptr;
  if (!h) {
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return fail(ctx_fail(c, GWAS_ERR_CUDA, "cusolverDnCreate failed"));
    sc.handles[c->device] = h;
  }
  cusolverDnSetStream(h, c->stream);
  ProfScope* eig_scope = new ProfScope(c, "eigendecomposition");
  const char* eig_env = std::getenv("GWAS_EIG");
  c->eig_steps = -1;
  rc = (eig_env && std::strcmp(eig_env, "fp64") == 0) ? EIG_FALL_BACK
                                                       : eig_refined(c, h, phi_d, n, c->Z, c->lam, &c->eig_steps);
  if (rc != GWAS_OK && rc != EIG_FALL_BACK) {
    delete eig_scope;
    return fail(rc);
  }
  int hinfo = 0;
  if (rc == EIG_FALL_BACK) {
    c->eig_steps = -1;
    int lwork = 0;
    if (cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, c->Z, n, c->lam, &lwork) !=
        CUSOLVER_STATUS_SUCCESS) {
      delete eig_scope;
      return fail(ctx_fail(c, GWAS_ERR_CUDA, "syevd workspace query failed"));
    }
    double* work = nullptr;
    int* info = nullptr;
    if ((rc = ctx_alloc(c, sizeof(double) * std::max(lwork, 1), (void**)&work)) ||
        (rc = ctx_alloc(c, sizeof(int), (void**)&info))) {
      delete eig_scope;
      return fail(rc);
    }
    cudaMemcpyAsync(c->Z, phi_d, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, c->stream);
    if (cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, c->Z, n, c->lam, work, lwork, info) !=
        CUSOLVER_STATUS_SUCCESS) {
      delete eig_scope;
      return fail(ctx_fail(c, GWAS_ERR_CUDA, "syevd failed to launch"));
    }
    if (!ctx_cuda_ok(c, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "info", &rc)) {
      delete eig_scope;
      return fail(rc);
    }
    ctx_free(c, work);
    ctx_free(c, info);
  }
  delete eig_scope;
  c->h_lam.resize(n);
  if (!ctx_cuda_ok(c, cudaMemcpyAsync(c->h_lam.data(), c->lam, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream),
                   "lambda", &rc))
    return fail(rc);
  if (!ctx_cuda_ok(c, cudaStreamSynchronize(c->stream), "eigendecomposition", &rc)) return fail(rc);
  solver_lock.unlock();
  ctx_free(c, phi_d);
  if (hinfo != 0) return fail(ctx_fail(c, GWAS_ERR_NOT_SPD, fmt("eigensolver did not converge (info %d)", hinfo)));
  for (double v : c->h_lam)
    if (!std::isfinite(v)) return fail(ctx_fail(c, GWAS_ERR_ARG, "Phi has non-finite entries"));

  // ---- heritabilities
  c->h_h2.assign(t, 0.0);
  {
    bool dev;
    if ((rc = ptr_kind(c, h2, &dev))) return fail(rc);
    if (dev) cudaMemcpy(c->h_h2.data(), h2, sizeof(double) * t, cudaMemcpyDeviceToHost);
    else std::memcpy(c->h_h2.data(), h2, sizeof(double) * t);
  }
  if ((rc = check_h2(c, c->h_h2))) return fail(rc);
  if ((rc = ctx_alloc(c, sizeof(double) * t, (void**)&c->h2))) return fail(rc);
  cudaMemcpyAsync(c->h2, c->h_h2.data(), sizeof(double) * t, cudaMemcpyHostToDevice, c->stream);

  // ---- covariates X_L and X'_L := Z^T X_L (Algorithm 5, gemm)
  if (pm1 > 0) {
    c->h_XL.resize((size_t)pm1 * n);
    bool dev;
    if ((rc = ptr_kind(c, XL, &dev))) return fail(rc);
    if (dev) cudaMemcpy(c->h_XL.data(), XL, sizeof(double) * pm1 * n, cudaMemcpyDeviceToHost);
    else std::memcpy(c->h_XL.data(), XL, sizeof(double) * pm1 * n);
    // X_L^T X_L and its inverse (full column rank is assumed by the paper, Section 2)
    std::vector<double> G(pm1 * pm1), L(pm1 * pm1, 0.0);
    for (int a = 0; a < pm1; ++a)
      for (int b = 0; b < pm1; ++b) {
        double s = 0;
        for (int k = 0; k < n; ++k) s += c->h_XL[(size_t)a * n + k] * c->h_XL[(size_t)b * n + k];
        G[a * pm1 + b] = s;
      }
    for (int a = 0; a < pm1; ++a)
      for (int b = 0; b <= a; ++b) {
        double s = G[a * pm1 + b];
        for (int k = 0; k < b; ++k) s -= L[a * pm1 + k] * L[b * pm1 + k];
        if (a == b) {
          if (!(s > 1e-12 * G[a * pm1 + a])) return fail(ctx_fail(c, GWAS_ERR_ARG, "X_L does not have full column rank"));
          L[a * pm1 + a] = std::sqrt(s);
        } else {
          L[a * pm1 + b] = s / L[b * pm1 + b];
        }
      }
    c->h_XtXinv.assign(pm1 * pm1, 0.0);
    for (int col = 0; col < pm1; ++col) {  // solve G x = e_col
      std::vector<double> z(pm1), x(pm1);
      for (int r = 0; r < pm1; ++r) {
        double s = (r == col);
        for (int k = 0; k < r; ++k) s -= L[r * pm1 + k] * z[k];
        z[r] = s / L[r * pm1 + r];
      }
      for (int r = pm1 - 1; r >= 0; --r) {
        double s = z[r];
        for (int k = r + 1; k < pm1; ++k) s -= L[k * pm1 + r] * x[k];
        x[r] = s / L[r * pm1 + r];
      }
      for (int r = 0; r < pm1; ++r) c->h_XtXinv[r * pm1 + col] = x[r];
    }
    if ((rc = ctx_alloc(c, sizeof(double) * pm1 * n, (void**)&c->XL))) return fail(rc);
    if ((rc = ctx_alloc(c, sizeof(double) * pm1 * n, (void**)&c->XLt))) return fail(rc);
    cudaMemcpyAsync(c->XL, c->h_XL.data(), sizeof(double) * pm1 * n, cudaMemcpyHostToDevice, c->stream);
    launch_rotate_fp64_rows(c, c->XL, pm1, n, c->XLt);
  }
  if (!ctx_cuda_ok(c, cudaStreamSynchronize(c->stream), "setup", &rc)) return fail(rc);
  if (!ctx_cuda_ok(c, cudaGetLastError(), "setup kernels", &rc)) return fail(rc);
  prof_flush(c);
  *out = c;
  return GWAS_OK;
}

extern "C" int gwas_set_h2(gwas_ctx* c, int t, const double* h2) {
  if (!c) return GWAS_ERR_ARG;
  if (t != c->t || !h2) return ctx_fail(c, GWAS_ERR_ARG, "t differs from setup or h2 is NULL");
  DeviceGuard guard(c->device);
  std::vector<double> v(t);
  bool dev;
  int rc = ptr_kind(c, h2, &dev);
  if (rc) return rc;
  if (dev) cudaMemcpy(v.data(), h2, sizeof(double) * t, cudaMemcpyDeviceToHost);
  else std::memcpy(v.data(), h2, sizeof(double) * t);
  if ((rc = check_h2(c, v))) return rc;
  c->h_h2 = v;
  ++c->h2_gen;  // plans that depend on the heritabilities (the interpolated S_BR) are redone
  cudaMemcpyAsync(c->h2, v.data(), sizeof(double) * t, cudaMemcpyHostToDevice, c->stream);
  if (!ctx_cuda_ok(c, cudaStreamSynchronize(c->stream), "set_h2", &rc)) return rc;
  return GWAS_OK;
}

extern "C" int gwas_load_snps(gwas_ctx* c, int64_t m, const int8_t* XR) {
  if (!c) return GWAS_ERR_ARG;
  if (m < 1 || !XR) return ctx_fail(c, GWAS_ERR_ARG, "m must be >= 1 and XR non-NULL");
  DeviceGuard guard(c->device);
  int rc = GWAS_OK;
  if (serve_busy(c)) return ctx_fail(c, GWAS_ERR_STATE, "gwas_load_snps while serving requests are pending");
  serve_shutdown(c);
  // drop previous genotypes
  ctx_free(c, c->Xt);
  c->Xt = nullptr;
  mixed_free(c);
  c->m = 0;
  bool dev;
  if ((rc = ptr_kind(c, XR, &dev))) return rc;
  const size_t bytes = (size_t)m * c->n;
  int8_t* dX = nullptr;
  // mixed path, page-locked host genotypes the device can read: the conversion kernel reads them
  // once and leaves the device copy the other kernels read
  const void* mapped = nullptr;
  const bool direct = !dev && c->precision == GWAS_MIXED && direct_host_input(c, XR, bytes, &mapped);
  if (dev) {
    dX = (int8_t*)XR;
  } else {
    if ((rc = ctx_alloc(c, bytes, (void**)&dX))) return rc;
    if (!direct &&
        !ctx_cuda_ok(c, cudaMemcpyAsync(dX, XR, bytes, cudaMemcpyHostToDevice, c->stream), "genotype upload", &rc)) {
      ctx_free(c, dX);
      return rc;
    }
  }
  if (c->precision == GWAS_FP64) {
    // X'_R := Z^T X_R (Algorithm 5, gemm), kept resident as [m][n] FP64
    if ((rc = ctx_alloc(c, sizeof(double) * m * c->n, (void**)&c->Xt)) == GWAS_OK)
      launch_rotate_fp64_i8(c, dX, m, c->n, c->Xt);
  } else if (direct) {
    rc = mixed_load(c, (const int8_t*)mapped, m, false, dX);
  } else {
    rc = mixed_load(c, dX, m);
  }
  if (rc == GWAS_OK) ctx_cuda_ok(c, cudaStreamSynchronize(c->stream), "load_snps", &rc);
  if (rc == GWAS_OK) ctx_cuda_ok(c, cudaGetLastError(), "load_snps kernels", &rc);
  if (!dev) ctx_free(c, dX);
  if (rc == GWAS_OK) prof_flush(c);
  if (rc == GWAS_OK) c->m = m;
  return rc;
}

namespace {

// Where the results of a trait block go.
struct OutSink {
  int kind = 0;           // 0: device array, 1: host array, 2: caller's host ring + callback
  void* out = nullptr;    // kinds 0 and 1: the full output array
  void* ring[2] = {nullptr, nullptr};
  gwas_block_fn fn = nullptr;
  void* user = nullptr;
};

int ensure_copy_stream(gwas_ctx* c) {
  int rc = GWAS_OK;
  if (!c->copy_stream &&
      !ctx_cuda_ok(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "copy stream", &rc))
    return rc;
  for (int k = 0; k < 2; ++k) {
    if (!c->ev_compute[k] &&
        !ctx_cuda_ok(c, cudaEventCreateWithFlags(&c->ev_compute[k], cudaEventDisableTiming), "event", &rc))
      return rc;
    if (!c->ev_copy[k] && !ctx_cuda_ok(c, cudaEventCreateWithFlags(&c->ev_copy[k], cudaEventDisableTiming), "event", &rc))
      return rc;
  }
  return GWAS_OK;
}

// Runs the loops of Algorithm 5 over SNPs [i0, i1) x all traits in trait blocks of tb.
// Host-bound results are double-buffered through two device staging buffers: the
// copy of block b to the host (on a side stream) overlaps the computation of block
// b+1 (Section 4's double buffering, applied to the output stream).
int run_blocks(gwas_ctx* c, const double* dY, int64_t i0, int64_t i1, int tb, const OutSink& sink) {
  const int n = c->n, t = c->t, p = c->p;
  const int64_t M = i1 - i0;
  // Trait blocks [bj0[b], bj0[b] + bnb[b]).  Into a host array the downloads bound the solve (the
  // device -> host link is slower than the compute per trait), so the first block is small and
  // each next block grows by 1.4x up to tb: the link starts early and stays busy, each block's
  // compute hiding under the previous block's download.  Otherwise uniform blocks of tb.
  std::vector<int> bj0, bnb;
  {
    const int unit = c->precision == GWAS_MIXED ? mixed_tt(c->pm1) : 16;
    int nb = (sink.kind == 1 && t > tb) ? std::min(tb, std::max(unit, (tb / 8) / unit * unit)) : tb;
    for (int j0 = 0; j0 < t;) {
      const int w = std::min(std::min(nb, tb), t - j0);  // never above tb: the workspaces hold tb traits
      bj0.push_back(j0);
      bnb.push_back(w);
      j0 += w;
      nb = std::min(tb, std::max(nb + unit, (int)(nb * 1.4) / unit * unit));
    }
  }
  const int nblocks = (int)bj0.size();
  const bool lastse = c->output == GWAS_OUT_LAST_SE;
  const size_t pair_bytes = lastse ? 2 * sizeof(float) : sizeof(double) * p;
  int rc = GWAS_OK;
  std::vector<void*> tmp;
  auto talloc = [&](size_t b, void** q) {
    int r = ctx_alloc(c, b, q);
    if (r == GWAS_OK) tmp.push_back(*q);
    return r;
  };
  MixedWs* ws = nullptr;
  double *Yt = nullptr, *R = nullptr, *cst = nullptr;
  void* stage[2] = {nullptr, nullptr};
  auto cleanup = [&]() {
    if (ws) mixed_ws_free(c, ws);
    for (void* q : tmp) ctx_free(c, q);
  };
  if (c->precision == GWAS_FP64) {
    if ((rc = talloc(sizeof(double) * tb * n, (void**)&Yt)) || (rc = talloc(sizeof(double) * tb * (p + 1) * n, (void**)&R)) ||
        (rc = talloc(sizeof(double) * tb * consts_stride(c->pm1), (void**)&cst))) {
      cleanup();
      return rc;
    }
  } else if ((rc = mixed_ws_alloc(c, tb, &ws))) {
    cleanup();
    return rc;
  }
  if (sink.kind != 0) {
    if ((rc = ensure_copy_stream(c)) || (rc = talloc(pair_bytes * (size_t)tb * M, &stage[0])) ||
        (rc = talloc(pair_bytes * (size_t)tb * M, &stage[1]))) {
      cleanup();
      return rc;
    }
  }
  // block b's device output pointers (beta or b, and se)
  auto block_out = [&](int b, int nb, void** ob, void** os) {
    const int j0 = bj0[b];
    *os = nullptr;
    if (sink.kind == 0) {
      if (!lastse) {
        *ob = (double*)sink.out + (size_t)j0 * M * p;
      } else {
        *ob = (float*)sink.out + (size_t)j0 * M;
        *os = (float*)sink.out + (size_t)t * M + (size_t)j0 * M;
      }
    } else {
      *ob = stage[b & 1];
      if (lastse) *os = (float*)stage[b & 1] + (size_t)nb * M;
    }
  };
  auto compute = [&](int b) -> int {
    const int j0 = bj0[b], nb = bnb[b];
    void *ob, *os;
    block_out(b, nb, &ob, &os);
    if (c->precision == GWAS_FP64) {
      launch_rotate_fp64_f64(c, dY + (size_t)j0 * n, nb, n, Yt);  // Y' := Z^T Y (gemm)
      launch_prep_fp64(c, Yt, nb, c->h2 + j0, R, cst);            // per-trait scalar-ops, syrk, gemv
      if (!lastse) {
        launch_fused_fp64(c, i0, i1, j0, nb, M, R, cst, ob);
      } else {
        void* pair[2] = {ob, os};
        launch_fused_fp64(c, i0, i1, j0, nb, M, R, cst, pair);
      }
      return GWAS_OK;
    }
    void* pair[2] = {ob, os};
    return mixed_solve_block(c, ws, dY + (size_t)j0 * n, j0, nb, i0, i1, M, lastse ? (void*)pair : ob);
  };
  auto copy_out = [&](int b) -> int {
    const int j0 = bj0[b], nb = bnb[b];
    const int k = b & 1;
    int r = GWAS_OK;
    // ev_compute[k] was recorded right after block b's kernels, so the download overlaps block b+1
    if (!ctx_cuda_ok(c, cudaStreamWaitEvent(c->copy_stream, c->ev_compute[k], 0), "event wait", &r)) return r;
    if (sink.kind == 2) {
      ctx_cuda_ok(c, cudaMemcpyAsync(sink.ring[k], stage[k], pair_bytes * (size_t)nb * M, cudaMemcpyDeviceToHost,
                                     c->copy_stream), "block download", &r);
    } else if (!lastse) {
      ctx_cuda_ok(c, cudaMemcpyAsync((double*)sink.out + (size_t)j0 * M * p, stage[k], sizeof(double) * p * nb * M,
                                     cudaMemcpyDeviceToHost, c->copy_stream), "block download", &r);
    } else {
      ctx_cuda_ok(c, cudaMemcpyAsync((float*)sink.out + (size_t)j0 * M, stage[k], sizeof(float) * nb * M,
                                     cudaMemcpyDeviceToHost, c->copy_stream), "block download", &r);
      if (r == GWAS_OK)
        ctx_cuda_ok(c, cudaMemcpyAsync((float*)sink.out + (size_t)t * M + (size_t)j0 * M, (float*)stage[k] + (size_t)nb * M,
                                       sizeof(float) * nb * M, cudaMemcpyDeviceToHost, c->copy_stream),
                    "block download", &r);
    }
    if (r == GWAS_OK) ctx_cuda_ok(c, cudaEventRecord(c->ev_copy[k], c->copy_stream), "event", &r);
    if (r == GWAS_OK && sink.kind == 2) {
      ctx_cuda_ok(c, cudaEventSynchronize(c->ev_copy[k]), "block download", &r);
      if (r == GWAS_OK) sink.fn(sink.user, j0, nb, sink.ring[k]);
    }
    return r;
  };
  for (int b = 0; b <= nblocks && rc == GWAS_OK; ++b) {
    if (b < nblocks) {
      // staging buffer b&1 was last read by the copy of block b-2
      if (sink.kind != 0 && b >= 2)
        ctx_cuda_ok(c, cudaStreamWaitEvent(c->stream, c->ev_copy[b & 1], 0), "event wait", &rc);
      if (rc == GWAS_OK) rc = compute(b);
      if (rc == GWAS_OK && sink.kind != 0)
        ctx_cuda_ok(c, cudaEventRecord(c->ev_compute[b & 1], c->stream), "event", &rc);
    }
    if (rc == GWAS_OK && sink.kind != 0 && b >= 1) rc = copy_out(b - 1);
  }
  if (rc == GWAS_OK) ctx_cuda_ok(c, cudaStreamSynchronize(c->stream), "solve", &rc);
  if (rc == GWAS_OK && c->copy_stream) ctx_cuda_ok(c, cudaStreamSynchronize(c->copy_stream), "solve copies", &rc);
  cleanup();
  return rc;
}

int solve_impl(gwas_ctx* c, const double* Y, int64_t i0, int64_t i1, int tb, const OutSink& sink) {
  int rc = GWAS_OK;
  c->singular = 0;
  const int64_t M = i1 - i0;
  if (M == 0) return GWAS_OK;
  const int n = c->n, t = c->t;
  bool ydev;
  if ((rc = ptr_kind(c, Y, &ydev))) return rc;
  cudaMemsetAsync(c->d_status, 0, 32, c->stream);
  double* yd = nullptr;
  const double* dY = Y;
  if (!ydev) {
    if ((rc = ctx_alloc(c, sizeof(double) * t * n, (void**)&yd))) return rc;
    if ((rc = ctx_upload(c, Y, sizeof(double) * t * n, yd))) {
      ctx_free(c, yd);
      return rc;
    }
    dY = yd;
  }
  rc = run_blocks(c, dY, i0, i1, tb, sink);
  unsigned long long st[2] = {0, 0};
  if (rc == GWAS_OK) ctx_cuda_ok(c, cudaGetLastError(), "solve kernels", &rc);
  if (rc == GWAS_OK) ctx_cuda_ok(c, cudaMemcpyAsync(st, c->d_status, 16, cudaMemcpyDeviceToHost, c->stream), "status", &rc);
  if (rc == GWAS_OK) ctx_cuda_ok(c, cudaStreamSynchronize(c->stream), "solve", &rc);
  if (rc == GWAS_OK) prof_flush(c);
  ctx_free(c, yd);
  if (rc) return rc;
  if (st[0]) return ctx_fail(c, GWAS_ERR_TIMEOUT, "a bounded wait inside a kernel ran out");
  c->singular = (int64_t)st[1];
  if (c->singular) return ctx_fail(c, GWAS_ERR_SINGULAR_PAIRS, fmt("%lld pairs with a singular system", (long long)st[1]));
  return GWAS_OK;
}

}  // namespace

extern "C" int gwas_solve(gwas_ctx* c, const double* Y, int64_t i0, int64_t i1, void* out) {
  if (!c) return GWAS_ERR_ARG;
  if (c->m == 0) return ctx_fail(c, GWAS_ERR_STATE, "gwas_solve before gwas_load_snps");
  if (!Y || !out) return ctx_fail(c, GWAS_ERR_ARG, "NULL Y or out");
  if (i0 < 0 || i1 < i0 || i1 > c->m) return ctx_fail(c, GWAS_ERR_ARG, "SNP range outside [0, m]");
  DeviceGuard guard(c->device);
  bool odev;
  int rc = ptr_kind(c, out, &odev);
  if (rc) return rc;
  OutSink sink;
  sink.kind = odev ? 0 : 1;
  sink.out = out;
  if (!odev) {
    // a page-locked host output that the device can address is written by the kernels
    // themselves, without device staging or copies
    const size_t pair_bytes = c->output == GWAS_OUT_LAST_SE ? 8 : 8 * (size_t)c->p;
    void* dptr = nullptr;
    if (direct_host_output(c, out, pair_bytes * (size_t)c->t * (size_t)(i1 - i0), &dptr)) {
      sink.kind = 0;
      sink.out = dptr;
      odev = true;
    }
  }
  int tb = (c->trait_block > 0 && c->trait_block < c->t) ? c->trait_block : c->t;
  if (!odev && c->trait_block <= 0 && i1 > i0) {
    // host output, no block size given: blocks of about 8 GB of results, so that the downloads
    // are pipelined behind the compute and the two staging buffers stay small
    const int64_t pair_bytes = c->output == GWAS_OUT_LAST_SE ? 8 : 8 * (int64_t)c->p;
    const int unit = c->precision == GWAS_MIXED ? mixed_tt(c->pm1) : 16;
    const int64_t per = (8ll << 30) / (pair_bytes * (i1 - i0));
    tb = (int)std::min<int64_t>(c->t, std::max<int64_t>(unit, per / unit * unit));
  }
  return solve_impl(c, Y, i0, i1, tb, sink);
}

extern "C" int gwas_solve_stream(gwas_ctx* c, const double* Y, int64_t i0, int64_t i1, int block_traits,
                                 void* host_buf0, void* host_buf1, gwas_block_fn fn, void* user) {
  if (!c) return GWAS_ERR_ARG;
  if (c->m == 0) return ctx_fail(c, GWAS_ERR_STATE, "gwas_solve_stream before gwas_load_snps");
  if (!Y || !host_buf0 || !host_buf1 || !fn || block_traits < 1)
    return ctx_fail(c, GWAS_ERR_ARG, "NULL argument or block_traits < 1");
  if (i0 < 0 || i1 < i0 || i1 > c->m) return ctx_fail(c, GWAS_ERR_ARG, "SNP range outside [0, m]");
  DeviceGuard guard(c->device);
  bool d0, d1;
  int rc;
  if ((rc = ptr_kind(c, host_buf0, &d0)) || (rc = ptr_kind(c, host_buf1, &d1))) return rc;
  if (d0 || d1) return ctx_fail(c, GWAS_ERR_ARG, "gwas_solve_stream buffers must be host memory");
  OutSink sink;
  sink.kind = 2;
  sink.ring[0] = host_buf0;
  sink.ring[1] = host_buf1;
  sink.fn = fn;
  sink.user = user;
  return solve_impl(c, Y, i0, i1, std::min(block_traits, c->t), sink);
}

// Out-of-core solve (Section 4: slabs of X_R through two buffers while the previous slab is
// processed).  The per-trait operands of every trait block are prepared once, up front.  Then
// units u = (slab s, trait block b), slab-major: the slab's conversion and rotation
// (gwas_load_snps' work, into slab-sized arrays) before its first block, and the fused kernel
// of every block into output staging k = u & 1.  Uploads of the next slab run on a stream of
// their own, downloads of finished pieces on the copy stream; the host calls fn per piece.
extern "C" int gwas_solve_ooc(gwas_ctx* c, int64_t m, const int8_t* XR, int64_t slab, const double* Y,
                              int block_traits, void* host_buf0, void* host_buf1, gwas_slab_fn fn, void* user) {
  if (!c) return GWAS_ERR_ARG;
  if (m < 1 || slab < 0 || block_traits < 1 || !XR || !Y || !host_buf0 || !host_buf1 || !fn)
    return ctx_fail(c, GWAS_ERR_ARG, "gwas_solve_ooc needs m >= 1, slab >= 0, block_traits >= 1 and non-NULL arguments");
  DeviceGuard guard(c->device);
  if (serve_busy(c)) return ctx_fail(c, GWAS_ERR_STATE, "gwas_solve_ooc while serving requests are pending");
  serve_shutdown(c);
  int rc;
  bool xdev, ydev, d0, d1;
  if ((rc = ptr_kind(c, XR, &xdev)) || (rc = ptr_kind(c, Y, &ydev)) || (rc = ptr_kind(c, host_buf0, &d0)) ||
      (rc = ptr_kind(c, host_buf1, &d1)))
    return rc;
  if (d0 || d1) return ctx_fail(c, GWAS_ERR_ARG, "gwas_solve_ooc buffers must be host memory");
  bool xpinned = false;
  if (!xdev) {
    cudaPointerAttributes at;
    xpinned = cudaPointerGetAttributes(&at, XR) == cudaSuccess && at.type == cudaMemoryTypeHost;
    cudaGetLastError();
  }
  // the slabs take the place of a resident genotype set
  ctx_free(c, c->Xt);
  c->Xt = nullptr;
  mixed_free(c);
  c->m = 0;
  c->singular = 0;
  const int n = c->n, t = c->t, p = c->p, q = c->pm1;
  if (slab == 0) slab = 1 << 20;
  slab = std::min<int64_t>((slab + 127) / 128 * 128, (m + 127) / 128 * 128);
  const int tb = std::min(block_traits, t);
  const int nblocks = (t + tb - 1) / tb;
  const int64_t nslabs = (m + slab - 1) / slab, U = nslabs * nblocks;
  const bool lastse = c->output == GWAS_OUT_LAST_SE, mixed = c->precision == GWAS_MIXED;
  const size_t pair_bytes = lastse ? 2 * sizeof(float) : sizeof(double) * p;
  std::vector<void*> tmp;
  auto talloc = [&](size_t b, void** ptr) {
    int r = ctx_alloc(c, b, ptr);
    if (r == GWAS_OK) tmp.push_back(*ptr);
    return r;
  };
  MixedWs* ws = nullptr;
  int8_t* hX[2] = {nullptr, nullptr};
  int8_t* dX[2] = {nullptr, nullptr};
  double *dY = (double*)Y, *Yt = nullptr, *R = nullptr, *cst = nullptr;
  __nv_bfloat16 *B1 = nullptr, *B2 = nullptr;
  float* cst32 = nullptr;
  void* stage[2] = {nullptr, nullptr};
  void* ring[2] = {host_buf0, host_buf1};
  cudaEvent_t ev_up[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
  cudaStream_t up = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(c->stream);
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    if (up) {
      cudaStreamSynchronize(up);
      cudaStreamDestroy(up);
    }
    if (ws) mixed_ws_free(c, ws);
    for (void* ptr : tmp) ctx_free(c, ptr);
    for (int k = 0; k < 2; ++k) {
      if (hX[k]) cudaFreeHost(hX[k]);
      if (ev_up[k]) cudaEventDestroy(ev_up[k]);
      if (ev_used[k]) cudaEventDestroy(ev_used[k]);
    }
    ctx_free(c, c->Xt);
    c->Xt = nullptr;
    mixed_free(c);
    c->m = 0;
  };
  auto fail = [&](int r) {
    cleanup();
    return r;
  };
  cudaMemsetAsync(c->d_status, 0, 32, c->stream);
  if (!ydev && ((rc = talloc(sizeof(double) * t * n, (void**)&dY)) || (rc = ctx_upload(c, Y, sizeof(double) * t * n, dY))))
    return fail(rc);
  if ((rc = ensure_copy_stream(c)) || (rc = talloc(pair_bytes * (size_t)tb * slab, &stage[0])) ||
      (rc = talloc(pair_bytes * (size_t)tb * slab, &stage[1])))
    return fail(rc);
  if (!ctx_cuda_ok(c, cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking), "upload stream", &rc)) return fail(rc);
  for (int k = 0; k < 2; ++k) {
    if (!ctx_cuda_ok(c, cudaEventCreateWithFlags(&ev_up[k], cudaEventDisableTiming), "event", &rc) ||
        !ctx_cuda_ok(c, cudaEventCreateWithFlags(&ev_used[k], cudaEventDisableTiming), "event", &rc))
      return fail(rc);
    if (!xdev && (rc = talloc((size_t)slab * n, (void**)&dX[k]))) return fail(rc);
    if (!xdev && !xpinned && cudaHostAlloc((void**)&hX[k], (size_t)slab * n, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      hX[k] = nullptr;
      return fail(ctx_fail(c, GWAS_ERR_OOM, "pinned staging of the genotype slabs"));
    }
  }
  // ---- the per-trait operands of every trait block, prepared once
  const int TT = mixed_tt(q), tm = fused_trait_tile_multiple();
  const int tpb = ((tb + TT - 1) / TT + tm - 1) / tm * tm;  // trait tiles allocated per block
  const int pair = mixed ? mixed_pair_layout(c) : 0;
  int64_t kp = 0;
  if (mixed) {
    if ((rc = mixed_ws_alloc(c, tb, &ws))) return fail(rc);
    kp = mixed_kpad(c);
    if ((rc = talloc(2ull * nblocks * c1_alloc_rows(q, tb) * kp, (void**)&B1)) ||
        (rc = talloc(2ull * nblocks * tpb * c2_alloc(q) * kp, (void**)&B2)) ||
        (rc = talloc(sizeof(float) * nblocks * tpb * TT * cst_stride(q), (void**)&cst32)))
      return fail(rc);
    cudaMemsetAsync(B1, 0, 2ull * nblocks * c1_alloc_rows(q, tb) * kp, c->stream);
    cudaMemsetAsync(B2, 0, 2ull * nblocks * tpb * c2_alloc(q) * kp, c->stream);
  } else if ((rc = talloc(sizeof(double) * tb * n, (void**)&Yt)) ||
             (rc = talloc(sizeof(double) * t * (p + 1) * n, (void**)&R)) ||
             (rc = talloc(sizeof(double) * t * consts_stride(q), (void**)&cst)) ||
             (rc = ctx_alloc(c, sizeof(double) * slab * n, (void**)&c->Xt))) {
    return fail(rc);
  }
  auto b1_of = [&](int b) { return B1 + (size_t)b * c1_alloc_rows(q, tb) * kp; };
  auto b2_of = [&](int b) { return B2 + (size_t)b * tpb * c2_alloc(q) * kp; };
  auto cst_of = [&](int b) { return cst32 + (size_t)b * tpb * TT * cst_stride(q); };
  for (int b = 0; b < nblocks && rc == GWAS_OK; ++b) {
    const int j0 = b * tb, nb = std::min(tb, t - j0);
    if (mixed) {
      // the layout of the kernel that runs this block (interpolated S_BR or contracted)
      const bool ip = mixed_block_interp(c, nb);
      rc = mixed_prep_traits(c, ws, dY + (size_t)j0 * n, c->h2 + j0, nb, b1_of(b), b2_of(b), cst_of(b), nullptr,
                             ip ? 0 : pair, ip ? tile_traits(q, true) : 0);
    } else {
      launch_rotate_fp64_f64(c, dY + (size_t)j0 * n, nb, n, Yt);
      launch_prep_fp64(c, Yt, nb, c->h2 + j0, R + (size_t)j0 * (p + 1) * n, cst + (size_t)j0 * consts_stride(q));
    }
  }
  if (rc) return fail(rc);
  // ---- slabs
  auto slab_rows = [&](int64_t s) { return std::min<int64_t>(slab, m - s * slab); };
  auto upload = [&](int64_t s) -> int {
    const int64_t rows = slab_rows(s);
    const int k = (int)(s & 1);
    int r = GWAS_OK;
    // int8 buffer k was last read by the conversion of slab s - 2
    if (s >= 2 && !ctx_cuda_ok(c, cudaStreamWaitEvent(up, ev_used[k], 0), "event wait", &r)) return r;
    const int8_t* src = XR + (size_t)(s * slab) * n;
    if (!xpinned) {
      // pinned staging k was last read by the upload of slab s - 2
      if (s >= 2 && !ctx_cuda_ok(c, cudaEventSynchronize(ev_up[k]), "slab upload", &r)) return r;
      std::memcpy(hX[k], src, (size_t)rows * n);
      src = hX[k];
    }
    if (ctx_cuda_ok(c, cudaMemcpyAsync(dX[k], src, (size_t)rows * n, cudaMemcpyHostToDevice, up), "slab upload", &r))
      ctx_cuda_ok(c, cudaEventRecord(ev_up[k], up), "event", &r);
    return r;
  };
  auto compute = [&](int64_t u) -> int {
    const int64_t s = u / nblocks, rows = slab_rows(s);
    const int b = (int)(u % nblocks), j0 = b * tb, nb = std::min(tb, t - j0), k = (int)(u & 1);
    int r = GWAS_OK;
    if (b == 0) {
      // the slab's conversion and rotation, then the next slab's upload
      const int ks = (int)(s & 1);
      const int8_t* xs = xdev ? XR + (size_t)(s * slab) * n : dX[ks];
      if (!xdev && !ctx_cuda_ok(c, cudaStreamWaitEvent(c->stream, ev_up[ks], 0), "event wait", &r)) return r;
      if (mixed) {
        if ((r = mixed_load(c, xs, rows, true))) return r;
      } else {
        launch_rotate_fp64_i8(c, xs, rows, n, c->Xt);
      }
      if (!xdev && !ctx_cuda_ok(c, cudaEventRecord(ev_used[ks], c->stream), "event", &r)) return r;
      if (!xdev && s + 1 < nslabs && (r = upload(s + 1))) return r;
    }
    // output staging k was last read by the download of unit u - 2
    if (u >= 2 && !ctx_cuda_ok(c, cudaStreamWaitEvent(c->stream, c->ev_copy[k], 0), "event wait", &r)) return r;
    void* pieces[2] = {stage[k], (float*)stage[k] + (size_t)nb * rows};
    void* out = lastse ? (void*)pieces : stage[k];
    if (mixed)
      r = mixed_fused_ops(c, b1_of(b), b2_of(b), cst_of(b), nb, 0, rows, rows, out, j0);
    else
      launch_fused_fp64(c, 0, rows, j0, nb, rows, R + (size_t)j0 * (p + 1) * n, cst + (size_t)j0 * consts_stride(q), out);
    // recorded here, not at delivery, so that the piece's download overlaps the next unit
    if (r == GWAS_OK) ctx_cuda_ok(c, cudaEventRecord(c->ev_compute[k], c->stream), "event", &r);
    return r;
  };
  auto deliver = [&](int64_t u) -> int {
    const int64_t s = u / nblocks, rows = slab_rows(s);
    const int b = (int)(u % nblocks), j0 = b * tb, nb = std::min(tb, t - j0), k = (int)(u & 1);
    int r = GWAS_OK;
    if (!ctx_cuda_ok(c, cudaStreamWaitEvent(c->copy_stream, c->ev_compute[k], 0), "event wait", &r) ||
        !ctx_cuda_ok(c, cudaMemcpyAsync(ring[k], stage[k], pair_bytes * (size_t)nb * rows, cudaMemcpyDeviceToHost,
                                        c->copy_stream), "piece download", &r) ||
        !ctx_cuda_ok(c, cudaEventRecord(c->ev_copy[k], c->copy_stream), "event", &r) ||
        !ctx_cuda_ok(c, cudaEventSynchronize(c->ev_copy[k]), "piece download", &r))
      return r;
    fn(user, s * slab, s * slab + rows, j0, nb, ring[k]);
    return GWAS_OK;
  };
  if (!xdev) rc = upload(0);
  for (int64_t u = 0; u <= U && rc == GWAS_OK; ++u) {
    if (u < U) rc = compute(u);
    if (rc == GWAS_OK && u >= 1) rc = deliver(u - 1);
  }
  unsigned long long st[2] = {0, 0};
  if (rc == GWAS_OK) ctx_cuda_ok(c, cudaGetLastError(), "solve kernels", &rc);
  if (rc == GWAS_OK) ctx_cuda_ok(c, cudaMemcpyAsync(st, c->d_status, 16, cudaMemcpyDeviceToHost, c->stream), "status", &rc);
  if (rc == GWAS_OK) ctx_cuda_ok(c, cudaStreamSynchronize(c->stream), "solve", &rc);
  if (rc == GWAS_OK) prof_flush(c);
  cleanup();
  if (rc) return rc;
  if (st[0]) return ctx_fail(c, GWAS_ERR_TIMEOUT, "a bounded wait inside a kernel ran out");
  c->singular = (int64_t)st[1];
  if (c->singular) return ctx_fail(c, GWAS_ERR_SINGULAR_PAIRS, fmt("%lld pairs with a singular system", (long long)st[1]));
  return GWAS_OK;
}
