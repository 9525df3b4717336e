// Serving: requests with their own traits (Y, h^2) and SNP ranges against the resident
// genotypes, processed with continuous batching.
//
// A scheduler thread owned by the context runs rounds.  Each round it
//   1. admits queued requests (first come, first served) while their trait tiles fit the
//      operand arena, whose size is the admission budget in HBM;
//   2. prepares the per-trait operands of the newly admitted requests (rotation of
//      their traits, per-trait algebra, back-rotation, slicing) into their arena slots;
//   3. builds a list of work units (one SNP tile x one trait tile of one request) and
//      runs the persistent fused kernel over the list.  The round is shared by remaining
//      size: every active request first gets a floor of round_units / (4 x active) units
//      (so that no request starves), then the rest of the round goes to the requests
//      with the fewest remaining units first, so a small request finishes in the round
//      after its arrival however large the requests beside it are;
//   4. marks the requests whose last unit ran as done and frees their slots.
// Requests that arrive while a round runs join the next one, so work of different
// requests overlaps on the device.  The arithmetic of a pair does not depend on which
// requests share its round, so results are the same alone and in a mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fused.cuh"
#include "gwas_internal.cuh"

namespace {

constexpr int GROUP = 16;  // SNP tiles per traversal group of a request

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t id = 0;
  int tk = 0;
  int64_t i0 = 0, i1 = 0;
  void* out = nullptr;
  std::vector<double> Y, h2;  // host copies until the operands are prepared
  int state = 0;              // 0 queued, 1 admitted, 2 done, 3 failed
  int rc = GWAS_OK;
  std::vector<int> slots;     // arena trait-tile slot of each trait tile
  int desc = -1;              // index in the device request table
  int64_t units = 0, next_unit = 0, done_units = 0;
  int nt = 0, ns = 0;         // trait tiles, SNP tiles
  double t_submit = 0, t_admit = 0, t_done = 0;
  int64_t singular = 0;
};

}  // namespace

struct ServeState {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::map<uint64_t, Request> reqs;
  std::vector<uint64_t> active;  // admitted, not finished (admission order)
  uint64_t next_id = 1;
  bool stop = false;
  std::thread thread;
  // device resources
  int slots = 0, max_prep = 0, round_units = 0, max_reqs = 0;
  int tt = 0, b1_rows = 0, b2_rows = 0, cstr = 0;  // trait-tile geometry for q = p - 1 (mixed_tt, c1_rows, ...)
  std::vector<int> free_slots;
  std::vector<int> free_desc;
  __nv_bfloat16 *B1 = nullptr, *B2 = nullptr;
  float* cst = nullptr;
  ServeDesc* d_desc = nullptr;
  unsigned long long* d_sing = nullptr;
  int4* d_units = nullptr;
  int4* h_units = nullptr;    // pinned
  double* d_Y = nullptr;
  double* d_h2 = nullptr;
  int* d_slot = nullptr;
  double* h_Y = nullptr;      // pinned staging of a prep batch
  double* h_h2 = nullptr;
  int* h_slot = nullptr;
  MixedWs* ws = nullptr;
  int failed = GWAS_OK;
  std::string fail_msg;
  int64_t rounds = 0;
  // the round's upload of its work list and its persistent kernel launch, captured once as a
  // CUDA graph (the launch reads the unit count from d_nunits) and replayed every round after
  int* d_nunits = nullptr;
  int* h_nunits = nullptr;    // pinned
  cudaGraphExec_t round_graph = nullptr;
  bool graph_failed = false;
  int64_t graph_rounds = 0;
};

namespace {

// The fused kernel's arguments for a serving round, but for the unit count.
FusedArgs round_args(gwas_ctx* c, ServeState* S) {
  FusedArgs a{};
  a.Kpad = (int)((c->n + 63) / 64 * 64);
  a.mpad = mixed_mpad(c);
  a.dof = (float)(c->n - c->p);
  a.sA = mixed_sA(c);
  a.acoef = mixed_acoef(c);
  a.cst = S->cst;
  a.status = c->d_status;
  a.singular = c->d_status + 1;
  a.units = S->d_units;
  a.reqs = S->d_desc;
  return a;
}

// Captures a round as a CUDA graph: the upload of the work list and its count from the pinned
// buffers, and the persistent kernel over at most round_units units.  Every pointer it holds
// lives as long as the serving state.  On failure the rounds keep launching directly.
void capture_round(gwas_ctx* c, ServeState* S) {
  FusedArgs a = round_args(c, S);
  a.nunits = S->round_units;
  a.nunits_dev = S->d_nunits;
  const bool prof = c->profile;
  const int64_t launches = c->launches;
  c->profile = false;  // no timing events inside the graph
  cudaGraph_t g = nullptr;
  int rc = GWAS_ERR_CUDA;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
    cudaMemcpyAsync(S->d_units, S->h_units, sizeof(int4) * S->round_units, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(S->d_nunits, S->h_nunits, sizeof(int), cudaMemcpyHostToDevice, c->stream);
    rc = launch_fused_serve(c, c->pm1, a, mixed_G(c), mixed_A2(c), S->B1, S->B2, S->slots);
    if (cudaStreamEndCapture(c->stream, &g) != cudaSuccess) rc = GWAS_ERR_CUDA;
  }
  c->profile = prof;
  c->launches = launches;
  if (rc == GWAS_OK && g && cudaGraphInstantiate(&S->round_graph, g, 0) != cudaSuccess) S->round_graph = nullptr;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (!S->round_graph) S->graph_failed = true;
}

// Unit u of a request in its traversal order: groups of GROUP SNP tiles x all trait tiles.
void unit_coords(const Request& r, int64_t u, int& st, int& tt) {
  const int64_t per_group = (int64_t)GROUP * r.nt;
  const int64_t g = u / per_group, w = u % per_group;
  const int g0 = (int)(g * GROUP);
  const int gs = std::min(GROUP, r.ns - g0);
  tt = (int)(w / gs);
  st = g0 + (int)(w % gs);
}

void fail_all(gwas_ctx* c, ServeState* S, int rc, const std::string& msg) {
  std::lock_guard<std::mutex> lk(S->mu);
  S->failed = rc;
  S->fail_msg = msg;
  for (auto& kv : S->reqs)
    if (kv.second.state < 2) {
      kv.second.state = 3;
      kv.second.rc = rc;
      kv.second.t_done = now_s();
    }
  S->active.clear();
  S->queue.clear();
  S->cv_done.notify_all();
  (void)c;
}

void serve_loop(gwas_ctx* c) {
  ServeState* S = c->serve;
  cudaSetDevice(c->device);
  MixedState* ms = c->mixed;
  (void)ms;
  const int n = c->n;
  while (true) {
    std::vector<uint64_t> admitted;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->active.empty(); });
      if (S->stop) return;
      // 1. admission: first come, first served, while trait tiles and descriptors are free
      while (!S->queue.empty()) {
        Request& r = S->reqs[S->queue.front()];
        if ((int)S->free_slots.size() < r.nt || S->free_desc.empty()) break;
        r.slots.assign(S->free_slots.end() - r.nt, S->free_slots.end());
        S->free_slots.resize(S->free_slots.size() - r.nt);
        r.desc = S->free_desc.back();
        S->free_desc.pop_back();
        r.state = 1;
        r.t_admit = now_s();
        admitted.push_back(r.id);
        S->active.push_back(r.id);
        S->queue.pop_front();
      }
    }
    // 2. per-trait operands of the admitted requests, in batches of up to max_prep traits
    //    (each request padded to whole trait tiles so that tiles never mix requests)
    int rc = GWAS_OK;
    {
      std::vector<std::pair<uint64_t, int>> todo;  // (request, first trait tile) pieces
      for (uint64_t id : admitted) {
        Request* r;
        {
          std::lock_guard<std::mutex> lk(S->mu);
          r = &S->reqs[id];
        }
        ServeDesc d{};
        d.i0 = r->i0;
        d.i1 = r->i1;
        d.ldo = r->i1 - r->i0;
        d.ntrait = r->tk;
        d.full_b = c->output == GWAS_OUT_FULL_B;
        if (d.full_b) {
          d.b64 = (double*)r->out;
        } else {
          d.beta = (float*)r->out;
          d.se = (float*)r->out + (size_t)r->tk * d.ldo;
        }
        d.singular = S->d_sing + r->desc;
        cudaMemcpyAsync(S->d_desc + r->desc, &d, sizeof d, cudaMemcpyHostToDevice, c->stream);
        cudaMemsetAsync(S->d_sing + r->desc, 0, sizeof(unsigned long long), c->stream);
        for (int t0 = 0; t0 < r->nt; ++t0) todo.push_back({id, t0});
      }
      size_t k = 0;
      while (k < todo.size() && rc == GWAS_OK) {
        int rows = 0, tiles = 0;
        cudaStreamSynchronize(c->stream);  // the pinned staging is reused by every batch
        const int TT = S->tt;
        while (k < todo.size() && rows + TT <= S->max_prep) {
          Request* r;
          {
            std::lock_guard<std::mutex> lk(S->mu);
            r = &S->reqs[todo[k].first];
          }
          const int t0 = todo[k].second;
          for (int j = 0; j < TT; ++j) {
            const int jj = t0 * TT + j;
            double* yrow = S->h_Y + (size_t)(rows + j) * n;
            if (jj < r->tk) {
              std::memcpy(yrow, r->Y.data() + (size_t)jj * n, sizeof(double) * n);
              S->h_h2[rows + j] = r->h2[jj];
            } else {
              std::memset(yrow, 0, sizeof(double) * n);
              S->h_h2[rows + j] = 0.5;
            }
          }
          S->h_slot[tiles] = r->slots[t0];
          rows += TT;
          ++tiles;
          ++k;
        }
        cudaMemcpyAsync(S->d_Y, S->h_Y, sizeof(double) * rows * n, cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(S->d_h2, S->h_h2, sizeof(double) * rows, cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(S->d_slot, S->h_slot, sizeof(int) * tiles, cudaMemcpyHostToDevice, c->stream);
        rc = mixed_prep_traits(c, S->ws, S->d_Y, S->d_h2, rows, S->B1, S->B2, S->cst, S->d_slot, 0);
      }
      for (uint64_t id : admitted) {
        std::lock_guard<std::mutex> lk(S->mu);
        Request& r = S->reqs[id];
        std::vector<double>().swap(r.Y);
        std::vector<double>().swap(r.h2);
      }
    }
    if (rc != GWAS_OK) {
      fail_all(c, S, rc, c->err);
      return;
    }
    // 3. round: a floor share for every active request, then the rest by fewest remaining units
    int nu = 0;
    std::vector<std::pair<uint64_t, int64_t>> took;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const int nact = (int)S->active.size();
      if (nact == 0) continue;
      const int64_t floor_share = std::max<int64_t>(1, S->round_units / (4 * (int64_t)nact));
      // admission order within equal remaining work (stable sort)
      std::vector<uint64_t> order(S->active);
      std::stable_sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) {
        const Request &ra = S->reqs[a], &rb = S->reqs[b];
        return ra.units - ra.next_unit < rb.units - rb.next_unit;
      });
      std::map<uint64_t, int64_t> taken;
      for (int pass = 0; pass < 2 && nu < S->round_units; ++pass) {
        for (uint64_t id : order) {
          Request& r = S->reqs[id];
          const int64_t want = pass == 0 ? floor_share : S->round_units - nu;
          const int64_t take = std::min<int64_t>({want, r.units - r.next_unit, (int64_t)S->round_units - nu});
          for (int64_t u = 0; u < take; ++u) {
            int st, tt;
            unit_coords(r, r.next_unit + u, st, tt);
            S->h_units[nu++] = make_int4((int)((r.i0 & ~(int64_t)127) + (int64_t)st * 128), r.slots[tt], r.desc, tt);
          }
          if (take > 0) taken[id] += take;
          r.next_unit += take;
          if (nu >= S->round_units) break;
        }
      }
      for (const auto& kv : taken) took.push_back(kv);
    }
    if (nu > 0) {
      *S->h_nunits = (int)nu;
      if (S->round_graph) {
        // the captured upload (the whole work-list buffer and the count) and persistent launch
        if (cudaGraphLaunch(S->round_graph, c->stream) != cudaSuccess) {
          cudaGetLastError();
          rc = GWAS_ERR_CUDA;
        }
        ++S->graph_rounds;
        c->launches++;
      } else {
        cudaMemcpyAsync(S->d_units, S->h_units, sizeof(int4) * nu, cudaMemcpyHostToDevice, c->stream);
        FusedArgs a = round_args(c, S);
        a.nunits = (int)nu;
        rc = launch_fused_serve(c, c->pm1, a, mixed_G(c), mixed_A2(c), S->B1, S->B2, S->slots);
      }
      cudaError_t e = cudaStreamSynchronize(c->stream);
      unsigned long long st0 = 0;
      if (rc == GWAS_OK && e == cudaSuccess) {
        cudaMemcpy(&st0, c->d_status, sizeof st0, cudaMemcpyDeviceToHost);
        if (st0) rc = GWAS_ERR_TIMEOUT;
      }
      if (e != cudaSuccess) {
        cudaGetLastError();
        rc = GWAS_ERR_CUDA;
      }
      if (rc != GWAS_OK) {
        fail_all(c, S, rc, rc == GWAS_ERR_TIMEOUT ? "a bounded wait inside the serving kernel ran out"
                                                  : std::string("serving round: ") + cudaGetErrorString(e));
        return;
      }
      ++S->rounds;
      prof_flush(c);
      // after one direct round (which also set the kernel's attributes), capture the round
      if (!S->round_graph && !S->graph_failed) capture_round(c, S);
    }
    // 4. completions
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const double t = now_s();
      for (auto& tk : took) {
        Request& r = S->reqs[tk.first];
        r.done_units += tk.second;
      }
      std::vector<uint64_t> still;
      for (uint64_t id : S->active) {
        Request& r = S->reqs[id];
        if (r.done_units >= r.units) {
          unsigned long long sing = 0;
          cudaMemcpy(&sing, S->d_sing + r.desc, sizeof sing, cudaMemcpyDeviceToHost);
          r.singular = (int64_t)sing;
          r.state = 2;
          r.t_done = t;
          for (int sl : r.slots) S->free_slots.push_back(sl);
          r.slots.clear();
          S->free_desc.push_back(r.desc);
        } else {
          still.push_back(id);
        }
      }
      S->active.swap(still);
      S->cv_done.notify_all();
    }
  }
}

int serve_init(gwas_ctx* c) {
  (void)0;
  if (c->serve) return c->serve->failed;
  if (c->precision != GWAS_MIXED) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "serving runs the mixed-precision path");
  if (!c->mixed || c->m == 0) return ctx_fail(c, GWAS_ERR_STATE, "serving needs loaded genotypes");
  ServeState* S = new ServeState;
  const int n = c->n;
  const int64_t Kpad = (n + 63) / 64 * 64;
  S->slots = 512;
  S->max_prep = 2048;
  S->round_units = 152 * 48;
  S->max_reqs = 4096;
  if (const char* e = getenv("GWAS_SERVE_SLOTS")) S->slots = std::max(8, atoi(e));
  if (const char* e = getenv("GWAS_SERVE_ROUND")) S->round_units = std::max(152, atoi(e));
  const int q = c->pm1, TT = mixed_tt(q);
  S->tt = TT;
  S->b1_rows = c1_rows(q);
  S->b2_rows = c2_rows(q);
  S->cstr = cst_stride(q);
  int rc;
  auto fail = [&](int code) {
    ctx_free(c, S->B1); ctx_free(c, S->B2); ctx_free(c, S->cst); ctx_free(c, S->d_desc); ctx_free(c, S->d_sing);
    ctx_free(c, S->d_units); ctx_free(c, S->d_Y); ctx_free(c, S->d_h2); ctx_free(c, S->d_slot);
    ctx_free(c, S->d_nunits);
    if (S->ws) mixed_ws_free(c, S->ws);
    if (S->h_units) cudaFreeHost(S->h_units);
    if (S->h_nunits) cudaFreeHost(S->h_nunits);
    if (S->h_Y) cudaFreeHost(S->h_Y);
    if (S->h_h2) cudaFreeHost(S->h_h2);
    if (S->h_slot) cudaFreeHost(S->h_slot);
    delete S;
    return code;
  };
  if ((rc = ctx_alloc(c, 2ull * S->slots * S->b1_rows * Kpad, (void**)&S->B1)) ||
      (rc = ctx_alloc(c, 2ull * S->slots * S->b2_rows * Kpad, (void**)&S->B2)) ||
      (rc = ctx_alloc(c, sizeof(float) * S->slots * TT * S->cstr, (void**)&S->cst)) ||
      (rc = ctx_alloc(c, sizeof(ServeDesc) * S->max_reqs, (void**)&S->d_desc)) ||
      (rc = ctx_alloc(c, sizeof(unsigned long long) * S->max_reqs, (void**)&S->d_sing)) ||
      (rc = ctx_alloc(c, sizeof(int4) * S->round_units, (void**)&S->d_units)) ||
      (rc = ctx_alloc(c, sizeof(int), (void**)&S->d_nunits)) ||
      (rc = ctx_alloc(c, sizeof(double) * S->max_prep * n, (void**)&S->d_Y)) ||
      (rc = ctx_alloc(c, sizeof(double) * S->max_prep, (void**)&S->d_h2)) ||
      (rc = ctx_alloc(c, sizeof(int) * S->max_prep / TT, (void**)&S->d_slot)) ||
      (rc = mixed_ws_alloc(c, S->max_prep, &S->ws)))
    return fail(rc);
  if (cudaHostAlloc((void**)&S->h_units, sizeof(int4) * S->round_units, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_Y, sizeof(double) * S->max_prep * n, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_h2, sizeof(double) * S->max_prep, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_slot, sizeof(int) * S->max_prep / TT, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_nunits, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx_fail(c, GWAS_ERR_OOM, "pinned host staging for serving"));
  }
  cudaMemsetAsync(S->B1, 0, 2ull * S->slots * S->b1_rows * Kpad, c->stream);
  cudaMemsetAsync(S->B2, 0, 2ull * S->slots * S->b2_rows * Kpad, c->stream);
  cudaMemsetAsync(c->d_status, 0, 32, c->stream);
  cudaStreamSynchronize(c->stream);
  for (int i = S->slots - 1; i >= 0; --i) S->free_slots.push_back(i);
  for (int i = S->max_reqs - 1; i >= 0; --i) S->free_desc.push_back(i);
  c->serve = S;
  S->thread = std::thread(serve_loop, c);
  return GWAS_OK;
}

}  // namespace

void serve_shutdown(gwas_ctx* c) {
  ServeState* S = c->serve;
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->thread.joinable()) S->thread.join();
  cudaStreamSynchronize(c->stream);
  ctx_free(c, S->B1); ctx_free(c, S->B2); ctx_free(c, S->cst); ctx_free(c, S->d_desc); ctx_free(c, S->d_sing);
  ctx_free(c, S->d_units); ctx_free(c, S->d_Y); ctx_free(c, S->d_h2); ctx_free(c, S->d_slot);
  ctx_free(c, S->d_nunits);
  if (S->round_graph) cudaGraphExecDestroy(S->round_graph);
  if (S->ws) mixed_ws_free(c, S->ws);
  cudaFreeHost(S->h_units);
  cudaFreeHost(S->h_nunits);
  cudaFreeHost(S->h_Y);
  cudaFreeHost(S->h_h2);
  cudaFreeHost(S->h_slot);
  delete S;
  c->serve = nullptr;
}

extern "C" int gwas_submit(gwas_ctx* c, const double* Y, int tk, const double* h2k, int64_t i0, int64_t i1, void* out,
                           uint64_t* req_id) {
  if (!c) return GWAS_ERR_ARG;
  if (!Y || !h2k || !out || !req_id || tk < 1) return ctx_fail(c, GWAS_ERR_ARG, "NULL argument or tk < 1");
  if (i0 < 0 || i1 <= i0 || i1 > c->m) return ctx_fail(c, GWAS_ERR_ARG, "SNP range outside [0, m] or empty");
  int dev0 = 0;
  cudaGetDevice(&dev0);
  cudaSetDevice(c->device);
  int rc = serve_init(c);
  cudaSetDevice(dev0);
  if (rc) return rc;
  ServeState* S = c->serve;
  const int TT = S->tt;
  if ((tk + TT - 1) / TT > S->slots)
    return ctx_fail(c, GWAS_ERR_OOM, "request has more traits than the serving operand arena holds");
  // output: device memory or page-locked host memory (the kernel writes it directly)
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, out) != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, GWAS_ERR_ARG, "serving output must be device or page-locked host memory");
  }
  if (at.type == cudaMemoryTypeUnregistered)
    return ctx_fail(c, GWAS_ERR_ARG, "serving output must be device or page-locked host memory");
  if (at.type == cudaMemoryTypeDevice && at.device != c->device)
    return ctx_fail(c, GWAS_ERR_ARG, "serving output on another device");
  Request r;
  r.tk = tk;
  r.i0 = i0;
  r.i1 = i1;
  r.out = out;
  r.Y.resize((size_t)tk * c->n);
  r.h2.resize(tk);
  bool ydev, hdev;
  if ((rc = ptr_kind(c, Y, &ydev)) || (rc = ptr_kind(c, h2k, &hdev))) return rc;
  if (ydev) cudaMemcpy(r.Y.data(), Y, sizeof(double) * r.Y.size(), cudaMemcpyDeviceToHost);
  else std::memcpy(r.Y.data(), Y, sizeof(double) * r.Y.size());
  if (hdev) cudaMemcpy(r.h2.data(), h2k, sizeof(double) * tk, cudaMemcpyDeviceToHost);
  else std::memcpy(r.h2.data(), h2k, sizeof(double) * tk);
  const double lmin = c->h_lam.front(), lmax = c->h_lam.back();
  for (int j = 0; j < tk; ++j) {
    const double h = r.h2[j];
    if (!(h >= 0.0 && h <= 1.0)) return ctx_fail(c, GWAS_ERR_ARG, "h2 outside [0, 1]");
    const double dmin = std::min(h * lmin + 1 - h, h * lmax + 1 - h), dmax = std::max(h * lmin + 1 - h, h * lmax + 1 - h);
    if (!(dmin > 1e-12 * dmax)) return ctx_fail(c, GWAS_ERR_NOT_SPD, "M_j not positive definite");
  }
  r.nt = (tk + TT - 1) / TT;
  // SNP tiles start on multiples of 128 (the x'^2 planes are stored by 128-SNP tile);
  // the SNPs of the first tile below i0 are computed and not written
  r.ns = (int)((i1 - (i0 & ~(int64_t)127) + 127) / 128);
  r.units = (int64_t)r.nt * r.ns;
  r.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->failed) return ctx_fail(c, S->failed, S->fail_msg);
    r.id = S->next_id++;
    *req_id = r.id;
    S->reqs.emplace(r.id, std::move(r));
    S->queue.push_back(*req_id);
  }
  S->cv_work.notify_one();
  return GWAS_OK;
}

extern "C" int gwas_poll(gwas_ctx* c, uint64_t id, int* done) {
  if (!c || !done) return GWAS_ERR_ARG;
  *done = 0;
  ServeState* S = c->serve;
  if (!S) return ctx_fail(c, GWAS_ERR_ARG, "unknown request");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return ctx_fail(c, GWAS_ERR_ARG, "unknown request");
  *done = it->second.state >= 2;
  if (it->second.state == 3) return it->second.rc;
  return it->second.state == 2 && it->second.singular ? GWAS_ERR_SINGULAR_PAIRS : GWAS_OK;
}

extern "C" int gwas_wait(gwas_ctx* c, uint64_t id, double timeout_s) {
  if (!c) return GWAS_ERR_ARG;
  ServeState* S = c->serve;
  if (!S) return ctx_fail(c, GWAS_ERR_ARG, "unknown request");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return ctx_fail(c, GWAS_ERR_ARG, "unknown request");
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s));
  if (!S->cv_done.wait_until(lk, deadline, [&] { return it->second.state >= 2; }))
    return ctx_fail(c, GWAS_ERR_TIMEOUT, "request not finished within the timeout");
  if (it->second.state == 3) return it->second.rc;
  if (it->second.singular)
    return ctx_fail(c, GWAS_ERR_SINGULAR_PAIRS, "request has pairs with a singular system (NaN outputs)");
  return GWAS_OK;
}

int serve_busy(gwas_ctx* c) {
  ServeState* S = c->serve;
  if (!S) return 0;
  std::lock_guard<std::mutex> lk(S->mu);
  return !S->queue.empty() || !S->active.empty();
}

extern "C" int gwas_request_times(gwas_ctx* c, uint64_t id, double* t_submit, double* t_admit, double* t_done) {
  if (!c || !c->serve) return GWAS_ERR_ARG;
  ServeState* S = c->serve;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return ctx_fail(c, GWAS_ERR_ARG, "unknown request");
  if (t_submit) *t_submit = it->second.t_submit;
  if (t_admit) *t_admit = it->second.t_admit;
  if (t_done) *t_done = it->second.t_done;
  return GWAS_OK;
}

extern "C" int gwas_serve_stats(const gwas_ctx* c, int64_t* rounds, int64_t* graph_rounds) {
  if (!c) return GWAS_ERR_ARG;
  const ServeState* S = c->serve;
  if (rounds) *rounds = S ? S->rounds : 0;
  if (graph_rounds) *graph_rounds = S ? S->graph_rounds : 0;
  return GWAS_OK;
}
