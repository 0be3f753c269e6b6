// C ABI of the McMg online solve (include/mcmg.h): context and allocation,
// setup (Algorithm 1), the V-cycle launcher (Algorithm 2, captured once per
// workspace as a CUDA graph), the synchronous solve and the request server.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstring>
#include <memory>
#include <unordered_map>

#include "mcmg_internal.cuh"

// ------------------------------------------------------------------ context --
struct Request {
  uint64_t ticket = 0;
  mcmg_handle_s* h = nullptr;
  const double2* f = nullptr;
  double2* u = nullptr;
  mcmg_solve_opts o{};
  mcmg::KrylovBlock* blk = nullptr;  // every right-hand side, V-cycles batched
  size_t bytes_needed = 0;
  std::chrono::steady_clock::time_point t_submit;
  mcmg_status status = MCMG_PENDING;
  mcmg_solve_info info{};
  std::string err;                   // message of a failure on the server thread
  cudaEvent_t ready = nullptr;       // recorded on the caller's stream at submit
  ~Request() {
    if (ready) cudaEventDestroy(ready);
  }
};

struct mcmg_ctx_s {
  int device = 0;
  size_t budget = 0;
  std::atomic<size_t> used{0};
  // server
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::unordered_map<uint64_t, Request*> finished;
  uint64_t next_ticket = 1;
  std::thread worker;
  bool stop = false;
  bool running = false;
  size_t max_queue = 4096;
  // cross-request batching (server thread): its stream, and the descriptors
  // of batched launches, staged in pinned memory and uploaded once per round
  cudaStream_t sst = nullptr;
  mcmg::TsField* fd_h = nullptr;
  mcmg::TsField* fd_d = nullptr;
  int fd_cap = 0;
  cudaEvent_t fd_ev = nullptr;       // the last upload has been read
  unsigned long long cohort_rounds = 0, cohort_members = 0;   // for reporting
  bool batching = true;              // cross-request batching of V-cycles
};

namespace mcmg {

static thread_local std::string g_last_error;
std::atomic<unsigned long long> g_launches{0};

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

mcmg_status cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? MCMG_ERR_OOM : MCMG_ERR_CUDA;
}

mcmg_status dev_alloc(mcmg_handle_s* h, DevArena& a, void** p, size_t bytes) {
  mcmg_ctx_s* c = h->ctx;
  bytes = (bytes + 255) & ~(size_t)255;
  if (c->budget) {
    size_t cur = c->used.load();
    if (cur + bytes > c->budget) {
      set_error("HBM budget exhausted: %zu used + %zu requested > %zu", cur, bytes, c->budget);
      return MCMG_ERR_OOM;
    }
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaMalloc");
  }
  c->used += bytes;
  a.ptrs.push_back(*p);
  a.bytes += bytes;
  return MCMG_OK;
}

void arena_free(mcmg_handle_s* h, DevArena& a) {
  for (void* p : a.ptrs) cudaFree(p);
  if (h && h->ctx) h->ctx->used -= a.bytes;
  a.ptrs.clear();
  a.bytes = 0;
}

// ------------------------------------------------------------ V-cycle work --
mcmg_status vwork_create(mcmg_handle_s* h, int nrhs, VWork** out) {
  VWork* w = new VWork();
  w->nrhs = nrhs;
  {
    mcmg_status s = dev_alloc(h, w->arena, (void**)&w->cells, 2 * sizeof(float2*));
    if (s != MCMG_OK) {
      vwork_destroy(h, w);
      return s;
    }
  }
  for (int l = 0; l < h->L; ++l) {
    const Level& L = h->lv[l];
    size_t b = sizeof(float2) * (size_t)L.g.nodes() * L.C * nrhs;
    mcmg_status s;
    if ((s = dev_alloc(h, w->arena, (void**)&w->r[l], b)) ||
        (s = dev_alloc(h, w->arena, (void**)&w->e[l], b)) ||
        (s = dev_alloc(h, w->arena, (void**)&w->e2[l], b)) ||
        (s = dev_alloc(h, w->arena, (void**)&w->t[l], b))) {
      vwork_destroy(h, w);
      return s;
    }
  }
  *out = w;
  return MCMG_OK;
}

void vwork_destroy(mcmg_handle_s* h, VWork* w) {
  if (!w) return;
  if (w->graph) cudaGraphExecDestroy(w->graph);
  for (auto& kv : w->sub) cudaGraphExecDestroy(kv.second.first);
  arena_free(h, w->arena);
  delete w;
}

// Whether a one-field V-cycle of h can take the lift and the projection
// inside its level-0 steps (see TsParams::r_cell).
static bool can_fuse_io(const mcmg_handle_s* h) {
  return h->L > 1 && h->lv[0].nu_post >= 1 && ts_fused_io_supported(h->lv[0]);
}

// The level sequence of Algorithm 2 on workspace w, nrhs fields, after r_1
// has been written to w->r[0].  Returns the buffer that holds e_1.  With
// `fused` (one field, can_fuse_io): level 0 reads the scalar r through
// w->cells[0] and lifts it, and its last post-smoothing step writes the
// projected e through w->cells[1]; *e1_out is then null.
static mcmg_status enqueue_levels(mcmg_handle_s* h, VWork* w, int nrhs, cudaStream_t st,
                                  float2** e1_out, bool fused = false) {
  const int L = h->L;
  float2* ecur[MCMG_MAX_LEVELS];
  const float2* const* rcell = w->cells;
  float2* const* zcell = w->cells + 1;
  for (int l = 0; l < L; ++l) {                       // down cycle
    const Level& lv = h->lv[l];
    const bool io = fused && l == 0;
    float2* cur = nullptr;
    for (int i = 0; i < lv.nu_pre; ++i) {
      float2* out = (cur == w->e[l]) ? w->e2[l] : w->e[l];
      if (io)
        MCMG_TRY(launch_smooth_ts_io(lv, i, rcell, h->lift, cur, out, nullptr, nullptr, 0, st));
      else
        MCMG_TRY(launch_smooth(lv, i, w->r[l], cur, out, 0, nrhs, st));
      cur = out;
    }
    if (!cur) {
      MCMG_CUDA(cudaMemsetAsync(w->e[l], 0, sizeof(float2) * lv.g.nodes() * lv.C * nrhs, st));
      cur = w->e[l];
    }
    ecur[l] = cur;
    if (l < L - 1) {                                  // residual + restriction
      if (io)
        MCMG_TRY(launch_smooth_ts_io(lv, 0, rcell, h->lift, cur, w->t[l], nullptr, nullptr, 1, st));
      else
        MCMG_TRY(launch_smooth(lv, 0, w->r[l], cur, w->t[l], 1, nrhs, st));
      MCMG_TRY(launch_restrict(lv, w->t[l], w->r[l + 1], nrhs, st));
    }
  }
  for (int l = L - 2; l >= 0; --l) {                  // up cycle
    const Level& lv = h->lv[l];
    const bool io = fused && l == 0;
    MCMG_TRY(launch_prolong_add(lv, ecur[l + 1], ecur[l], nrhs, st));
    for (int i = 0; i < lv.nu_post; ++i) {
      float2* out = (ecur[l] == w->e[l]) ? w->e2[l] : w->e[l];
      if (io) {
        const bool last = i == lv.nu_post - 1;
        MCMG_TRY(launch_smooth_ts_io(lv, lv.nu_pre + i, rcell, h->lift, ecur[l], out,
                                     last ? zcell : nullptr, last ? h->proj : nullptr, 0, st));
      } else {
        MCMG_TRY(launch_smooth(lv, lv.nu_pre + i, w->r[l], ecur[l], out, 0, nrhs, st));
      }
      ecur[l] = out;
    }
  }
  *e1_out = fused ? nullptr : ecur[0];
  return MCMG_OK;
}

// Capture the level sequence for `count` fields of workspace w as a graph.
static mcmg_status capture_levels_n(mcmg_handle_s* h, VWork* w, int count, cudaGraphExec_t* exec,
                                    unsigned long long* kernels, bool fused = false) {
  cudaStream_t cs;
  MCMG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  float2* e1 = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  const unsigned long long before = g_launches.load();
  mcmg_status s = enqueue_levels(h, w, count, cs, &e1, fused);
  *kernels = g_launches.load() - before;
  g_launches.fetch_sub(*kernels);   // counted when the graph runs
  e = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (s != MCMG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  if (!fused) w->e1 = e1;
  return MCMG_OK;
}

// Drop graphs captured before a smoothing shape was overridden.
static void refresh_graphs(mcmg_handle_s* h, VWork* w) {
  if (w->shape_gen == h->shape_gen) return;
  if (w->graph) cudaGraphExecDestroy(w->graph);
  w->graph = nullptr;
  w->graph_fused = false;
  for (auto& kv : w->sub) cudaGraphExecDestroy(kv.second.first);
  w->sub.clear();
  w->shape_gen = h->shape_gen;
}

// The graph of all w->nrhs fields, captured fused or not as asked (a graph
// of the other kind is dropped first).
static mcmg_status ensure_graph(mcmg_handle_s* h, VWork* w, bool fused) {
  if (w->graph && w->graph_fused != fused) {
    cudaGraphExecDestroy(w->graph);
    w->graph = nullptr;
  }
  if (!w->graph) {
    MCMG_TRY(capture_levels_n(h, w, w->nrhs, &w->graph, &w->graph_kernels, fused));
    w->graph_fused = fused;
  }
  return MCMG_OK;
}

__global__ void k_set_cells(float2** cells, const float2* r, float2* e) {
  cells[0] = const_cast<float2*>(r);
  cells[1] = e;
}

mcmg_status vcycle_run_batch(mcmg_handle_s* h, VWork* w, const float2* const* srcs,
                             float2* const* dsts, int count, cudaStream_t st) {
  if (count < 1 || count > w->nrhs) {
    set_error("batch of %d fields in a workspace of %d", count, w->nrhs);
    return MCMG_ERR_ARG;
  }
  const Level& l0 = h->lv[0];
  refresh_graphs(h, w);
  MCMG_TRY(launch_lift_gather(srcs, h->lift, w->r[0], l0.C, l0.g.nodes(), count, st));
  cudaGraphExec_t exec;
  unsigned long long kernels;
  if (count == w->nrhs) {
    MCMG_TRY(ensure_graph(h, w, false));
    exec = w->graph;
    kernels = w->graph_kernels;
  } else {
    auto it = w->sub.find(count);
    if (it == w->sub.end()) {
      cudaGraphExec_t ex;
      unsigned long long kn;
      MCMG_TRY(capture_levels_n(h, w, count, &ex, &kn));
      it = w->sub.emplace(count, std::make_pair(ex, kn)).first;
    }
    exec = it->second.first;
    kernels = it->second.second;
  }
  MCMG_CUDA(cudaGraphLaunch(exec, st));
  count_launch(kernels);
  MCMG_TRY(launch_project_scatter(w->e1, h->proj, dsts, l0.C, l0.g.nodes(), count, st));
  return MCMG_OK;
}

mcmg_status vcycle_run(mcmg_handle_s* h, VWork* w, const float2* r, float2* e, int nrhs,
                       cudaStream_t st) {
  if (nrhs != w->nrhs) {
    set_error("workspace holds %d fields, call asks for %d", w->nrhs, nrhs);
    return MCMG_ERR_ARG;
  }
  const Level& l0 = h->lv[0];
  refresh_graphs(h, w);
  const bool fused = nrhs == 1 && can_fuse_io(h);
  if (fused) {
    // level 0 lifts r and projects e itself: only their addresses change
    k_set_cells<<<1, 1, 0, st>>>(w->cells, r, e);
    MCMG_CHECK_LAUNCH("set_cells");
  } else {
    MCMG_TRY(launch_lift(r, h->lift, w->r[0], l0.C, l0.g.nodes(), nrhs, st));
  }
  MCMG_TRY(ensure_graph(h, w, fused));
  MCMG_CUDA(cudaGraphLaunch(w->graph, st));
  count_launch(w->graph_kernels);
  if (!fused) MCMG_TRY(launch_project(w->e1, h->proj, e, l0.C, l0.g.nodes(), nrhs, st));
  return MCMG_OK;
}

}  // namespace mcmg

using namespace mcmg;

// ------------------------------------------------------------- entry points --
// (C linkage comes from the declarations in mcmg.h)

const char* mcmg_last_error(void) { return g_last_error.c_str(); }
const char* mcmg_version(void) { return "mcmg-b300 0.1 (sm_103a)"; }
uint64_t mcmg_kernel_launches(void) { return g_launches.load(); }

mcmg_status mcmg_ctx_create(int device, size_t hbm_budget_bytes, mcmg_ctx* out) {
  if (!out) { set_error("out is NULL"); return MCMG_ERR_ARG; }
  int ndev = 0;
  MCMG_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) {
    set_error("device %d out of range (%d devices)", device, ndev);
    return MCMG_ERR_ARG;
  }
  MCMG_CUDA(cudaSetDevice(device));
  mcmg_ctx_s* c = new mcmg_ctx_s();
  c->device = device;
  c->budget = hbm_budget_bytes;
  *out = c;
  return MCMG_OK;
}

static void server_stop(mcmg_ctx_s* c);

mcmg_status mcmg_ctx_destroy(mcmg_ctx c) {
  if (!c) return MCMG_OK;
  server_stop(c);
  for (auto& kv : c->finished) delete kv.second;
  delete c;
  return MCMG_OK;
}

mcmg_status mcmg_ctx_memory(mcmg_ctx c, size_t* used) {
  if (!c || !used) { set_error("NULL argument"); return MCMG_ERR_ARG; }
  *used = c->used.load();
  return MCMG_OK;
}

static bool pow2_channels(int C) {
  return C == 1 || C == 2 || C == 4 || C == 8 || C == 16 || C == 32 || C == 64;
}

// Reads the weight blob into device layouts.  See mcmg.h for the order.
struct BlobReader {
  const double* p;
  size_t left;
  bool ok = true;
  const double* take(size_t n) {
    if (n > left) { ok = false; return nullptr; }
    const double* r = p;
    p += n;
    left -= n;
    return r;
  }
};

static std::vector<float> to_f32(const double* src, size_t n) {
  std::vector<float> v(n);
  for (size_t i = 0; i < n; ++i) v[i] = (float)src[i];
  return v;
}

// complex M[b][co][ci] (nb blocks) -> float2 M^T[b][ci][co]
static std::vector<float2> transpose_blocks(const double* src, int nb, int co_n, int ci_n) {
  std::vector<float2> v((size_t)nb * co_n * ci_n);
  for (int b = 0; b < nb; ++b)
    for (int co = 0; co < co_n; ++co)
      for (int ci = 0; ci < ci_n; ++ci) {
        const double* s = src + 2 * (((size_t)b * co_n + co) * ci_n + ci);
        v[((size_t)b * ci_n + ci) * co_n + co] = make_float2((float)s[0], (float)s[1]);
      }
  return v;
}

// Host -> device upload ordered on the setup stream st.  A synchronous
// cudaMemcpy from pageable memory returns once the data is staged, and the
// setup kernels run on a non-blocking stream that does not wait for the
// legacy stream's copy: with the GPU busy (other requests' solves) a kernel
// could read the buffer before the copy had landed.  cudaMemcpyAsync on st
// orders the copy before the kernels that read it (the pageable source is
// staged before the call returns, so it may be released at once).
template <typename T>
static mcmg_status upload(mcmg_handle_s* h, DevArena& a, const std::vector<T>& v, T** out,
                          cudaStream_t st) {
  MCMG_TRY(dev_alloc(h, a, (void**)out, sizeof(T) * std::max<size_t>(v.size(), 1)));
  MCMG_CUDA(cudaMemcpyAsync(*out, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return MCMG_OK;
}

static mcmg_status setup_impl(mcmg_ctx c, const mcmg_medium* m, double omega,
                              const mcmg_weights* w, mcmg_handle_s* h) {
  const int d = m->dim;
  const int L = w->levels;
  Grid g0;
  g0.d = d;
  if (d == 2) { g0.ny = m->n[0]; g0.nx = m->n[1]; g0.nz = 1; }
  else { g0.nz = m->n[0]; g0.ny = m->n[1]; g0.nx = m->n[2]; }
  const int T = 2 * d + 1, T3 = d == 3 ? 27 : 9;
  h->g0 = g0;
  h->L = L;
  h->precision = w->precision;
  // batching key (coarse; every batched launch also checks the level
  // signatures below)
  h->wsig = ((uint64_t)w->precision << 8) | (uint64_t)d;
  // shapes
  Grid g = g0;
  for (int l = 0; l < L; ++l) {
    if (!pow2_channels(w->channels[l])) {
      set_error("channels[%d] = %d not in {1,2,4,8,16,32,64}", l, w->channels[l]);
      return MCMG_ERR_SHAPE;
    }
    if (g.nx < 2 || g.ny < 2 || (d == 3 && g.nz < 2)) {
      set_error("level %d grid smaller than 2 nodes per axis", l);
      return MCMG_ERR_SHAPE;
    }
    if (l < L - 1 && ((g.nx | g.ny | (d == 3 ? g.nz : 0)) & 1)) {
      set_error("level %d grid %dx%dx%d not divisible by 2", l, g.nz, g.ny, g.nx);
      return MCMG_ERR_SHAPE;
    }
    if (w->nu_pre[l] < 0 || w->nu_post[l] < 0 || (l == L - 1 && w->nu_post[l] != 0)) {
      set_error("bad smoothing counts on level %d", l);
      return MCMG_ERR_ARG;
    }
    h->lv[l].g = g;
    h->lv[l].C = w->channels[l];
    h->lv[l].Cn = l < L - 1 ? w->channels[l + 1] : 0;
    h->lv[l].nu_pre = w->nu_pre[l];
    h->lv[l].nu_post = w->nu_post[l];
    g = g.coarse();
  }
  // ---- parse the blob
  BlobReader br{w->blob, w->blob_len};
  const int C0 = w->channels[0];
  const double* flw = br.take((size_t)2 * C0 * 2 * T3);
  const double* flb = br.take((size_t)2 * C0);
  struct LvBlob { const double *W, *KA, *KS, *Ws, *fsw, *fsb, *R, *P, *faw, *fab; };
  std::vector<LvBlob> lb(L);
  for (int l = 0; l < L; ++l) {
    const int C = w->channels[l];
    const int ns = w->nu_pre[l] + w->nu_post[l];
    lb[l].W = br.take((size_t)2 * T * C * C);
    lb[l].KA = br.take((size_t)2 * C * C);
    lb[l].KS = br.take((size_t)2 * C * C);
    lb[l].Ws = br.take((size_t)2 * ns * C * C);
    lb[l].fsw = br.take((size_t)2 * C * 2 * C * T3);
    lb[l].fsb = br.take((size_t)2 * C);
    if (l < L - 1) {
      const int Cn = w->channels[l + 1];
      lb[l].R = br.take((size_t)2 * T3 * Cn * C);
      lb[l].P = br.take((size_t)2 * T3 * C * Cn);
      lb[l].faw = br.take((size_t)2 * Cn * 2 * C * T3);
      lb[l].fab = br.take((size_t)2 * Cn);
    }
  }
  const double* gl = br.take((size_t)2 * C0);
  const double* gp = br.take((size_t)2 * C0);
  if (!br.ok || br.left != 0) {
    set_error("weight blob length %zu does not match the model (%s)", w->blob_len,
              br.ok ? "too long" : "too short");
    return MCMG_ERR_ARG;
  }
  cudaStream_t st = h->stream;
  // ---- medium -> q
  const long long N = g0.nodes();
  DevArena tmp;
  double* c_dev = nullptr;
  auto cleanup = [&]() { arena_free(h, tmp); };
  mcmg_status s;
  if ((s = dev_alloc(h, tmp, (void**)&c_dev, sizeof(double) * N))) return cleanup(), s;
  MCMG_CUDA(cudaMemcpyAsync(c_dev, m->c, sizeof(double) * N, cudaMemcpyHostToDevice, st));
  if ((s = dev_alloc(h, h->arena, (void**)&h->q32, sizeof(float2) * N))) return cleanup(), s;
  if ((s = dev_alloc(h, h->arena, (void**)&h->q64, sizeof(double2) * N))) return cleanup(), s;
  if ((s = launch_make_q(c_dev, omega, m->sponge_width, m->gamma_max, g0, h->q32, h->q64, st)))
    return cleanup(), s;
  if ((s = dev_alloc(h, h->arena, (void**)&h->qdf, sizeof(float4) * N)) ||
      (s = launch_make_qdf(h->q64, h->qdf, g0, st)))
    return cleanup(), s;
  // ---- weights to device layouts
  for (int l = 0; l < L; ++l) {
    Level& lv = h->lv[l];
    const int C = lv.C, ns = lv.nu_pre + lv.nu_post;
    {
      auto fnv = [](uint64_t x, const void* data, size_t bytes) {
        const unsigned char* b = (const unsigned char*)data;
        for (size_t i = 0; i < bytes; ++i) x = (x ^ b[i]) * 1099511628211ull;
        return x;
      };
      uint64_t base = 1469598103934665603ull;
      base = fnv(base, &w->precision, sizeof(int));
      base = fnv(base, &C, sizeof(int));
      base = fnv(base, lb[l].W, sizeof(double) * 2 * T * C * C);
      base = fnv(base, lb[l].KA, sizeof(double) * 2 * C * C);
      lv.rsig = base;
      base = fnv(base, lb[l].KS, sizeof(double) * 2 * C * C);
      for (int i = 0; i < ns && i < 2 * 8 + 1; ++i)
        lv.ssig[i] = fnv(base, lb[l].Ws + (size_t)2 * i * C * C, sizeof(double) * 2 * C * C);
    }
    if ((s = upload(h, h->arena, transpose_blocks(lb[l].W, T, C, C), &lv.Wt, st)) ||
        (s = upload(h, h->arena, transpose_blocks(lb[l].KA, 1, C, C), &lv.KAt, st)) ||
        (s = upload(h, h->arena, transpose_blocks(lb[l].KS, 1, C, C), &lv.KSt, st)) ||
        (s = upload(h, h->arena, transpose_blocks(lb[l].Ws, std::max(ns, 1), C, C), &lv.Wsmt, st)))
      return cleanup(), s;
    if (l < L - 1) {
      const int Cn = lv.Cn;
      if ((s = upload(h, h->arena, transpose_blocks(lb[l].R, T3, Cn, C), &lv.Rt, st)) ||
          (s = upload(h, h->arena, transpose_blocks(lb[l].P, T3, C, Cn), &lv.Pt, st)))
        return cleanup(), s;
    }
    if ((s = dev_alloc(h, h->arena, (void**)&lv.a, sizeof(float2) * lv.g.nodes() * C)) ||
        (s = dev_alloc(h, h->arena, (void**)&lv.s, sizeof(float2) * lv.g.nodes() * C)))
      return cleanup(), s;
    lv.err = h->err_dev;
    if (w->precision == MCMG_BF16 && ts_supported(C, MCMG_BF16)) {
      // BF16 block forms of every matrix: taps, K_A, K_S, W^(i)
      const int K2 = 2 * C;
      const size_t tile = (size_t)K2 * K2;          // bf16 elements per matrix
      const int ntile = T + 2 + ns;
      std::vector<uint16_t> host(tile * ntile);
      std::vector<float2> mat((size_t)C * C);
      auto put = [&](const double* src, int t) {
        for (size_t i = 0; i < (size_t)C * C; ++i)
          mat[i] = make_float2((float)src[2 * i], (float)src[2 * i + 1]);
        pack_ts_bf16(mat.data(), C, host.data() + tile * t);
      };
      for (int t = 0; t < T; ++t) put(lb[l].W + (size_t)2 * t * C * C, t);
      put(lb[l].KA, T);
      put(lb[l].KS, T + 1);
      for (int i = 0; i < ns; ++i) put(lb[l].Ws + (size_t)2 * i * C * C, T + 2 + i);
      uint4* dst = nullptr;
      if ((s = dev_alloc(h, h->arena, (void**)&dst, host.size() * sizeof(uint16_t))))
        return cleanup(), s;
      MCMG_CUDA(cudaMemcpyAsync(dst, host.data(), host.size() * sizeof(uint16_t),
                                cudaMemcpyHostToDevice, st));
      lv.use_ts = true;
      lv.ts_prec = MCMG_BF16;
      lv.ts_mats = dst;
    }
    if (w->precision == MCMG_FP32_TC && ts_supported(C, MCMG_FP32_TC)) {
      // TF32 hi / lo halves of every matrix: taps, K_A, K_S, W^(i)
      const size_t per = (size_t)2 * (2 * C) * (2 * C);    // floats per matrix
      const int ntile = T + 2 + ns;
      std::vector<float> host(per * ntile);
      std::vector<float2> mat((size_t)C * C);
      auto put = [&](const double* src, int t) {
        for (size_t i = 0; i < (size_t)C * C; ++i)
          mat[i] = make_float2((float)src[2 * i], (float)src[2 * i + 1]);
        pack_ts_tf32(mat.data(), C, host.data() + per * t);
      };
      for (int t = 0; t < T; ++t) put(lb[l].W + (size_t)2 * t * C * C, t);
      put(lb[l].KA, T);
      put(lb[l].KS, T + 1);
      for (int i = 0; i < ns; ++i) put(lb[l].Ws + (size_t)2 * i * C * C, T + 2 + i);
      uint4* dst = nullptr;
      if ((s = dev_alloc(h, h->arena, (void**)&dst, host.size() * sizeof(float))))
        return cleanup(), s;
      MCMG_CUDA(cudaMemcpyAsync(dst, host.data(), host.size() * sizeof(float),
                                cudaMemcpyHostToDevice, st));
      lv.use_ts = true;
      lv.ts_prec = MCMG_FP32_TC;
      lv.ts_mats = dst;
    }
    if (lv.use_ts && l < L - 1) {
      // restriction R_o (Cn x C) and prolongation P_o (C x Cn), every tap
      const int Cn = lv.Cn;
      const bool tf = lv.ts_prec == MCMG_FP32_TC;
      const size_t per = (tf ? 2 * sizeof(float) : sizeof(uint16_t)) * (size_t)(2 * C) * (2 * Cn);
      std::vector<unsigned char> hr(per * T3), hp(per * T3);
      std::vector<float2> mat((size_t)C * Cn);
      if (C == 8) {
        // restriction from 8 channels runs two taps per stage: matrix k is
        // [R_2k | R_2k+1] (Cn x 16, the second zero past the last tap)
        const int npair = (T3 + 1) / 2;
        const size_t per2 = (tf ? 2 * sizeof(float) : sizeof(uint16_t)) * (size_t)32 * (2 * Cn);
        hr.assign(per2 * npair, 0);
        std::vector<float2> pm((size_t)Cn * 16);
        for (int k = 0; k < npair; ++k) {
          for (int co = 0; co < Cn; ++co)
            for (int ci = 0; ci < 16; ++ci) {
              const int t = 2 * k + (ci >> 3);
              const double* rs = lb[l].R + (size_t)2 * ((size_t)t * Cn * C + (size_t)co * C + (ci & 7));
              pm[(size_t)co * 16 + ci] =
                  t < T3 ? make_float2((float)rs[0], (float)rs[1]) : make_float2(0.f, 0.f);
            }
          pack_ts_rect(pm.data(), Cn, 16, tf, hr.data() + per2 * k);
        }
        // and, for the line-staged kernel, three taps per stage: matrix k is
        // [R_3k | R_3k+1 | R_3k+2] (o_x = -1, 0, +1 of stage (o_y, o_z) = k)
        const int nst = T3 / 3;
        const size_t per3 = (tf ? 2 * sizeof(float) : sizeof(uint16_t)) * (size_t)48 * (2 * Cn);
        std::vector<unsigned char> h3(per3 * nst, 0);
        std::vector<float2> tm((size_t)Cn * 24);
        for (int k = 0; k < nst; ++k) {
          for (int co = 0; co < Cn; ++co)
            for (int ci = 0; ci < 24; ++ci) {
              const int t = 3 * k + ci / 8;
              const double* rs = lb[l].R + (size_t)2 * ((size_t)t * Cn * C + (size_t)co * C + ci % 8);
              tm[(size_t)co * 24 + ci] = make_float2((float)rs[0], (float)rs[1]);
            }
          pack_ts_rect(tm.data(), Cn, 24, tf, h3.data() + per3 * k);
        }
        uint4* d3 = nullptr;
        if ((s = dev_alloc(h, h->arena, (void**)&d3, h3.size()))) return cleanup(), s;
        MCMG_CUDA(cudaMemcpyAsync(d3, h3.data(), h3.size(), cudaMemcpyHostToDevice, st));
        lv.ts_R3 = d3;
      }
      for (int t = 0; t < T3; ++t) {
        const double* rs = lb[l].R + (size_t)2 * t * Cn * C;
        for (size_t i = 0; i < (size_t)C * Cn; ++i)
          mat[i] = make_float2((float)rs[2 * i], (float)rs[2 * i + 1]);
        if (C != 8) pack_ts_rect(mat.data(), Cn, C, tf, hr.data() + per * t);
        const double* ps = lb[l].P + (size_t)2 * t * C * Cn;
        for (size_t i = 0; i < (size_t)C * Cn; ++i)
          mat[i] = make_float2((float)ps[2 * i], (float)ps[2 * i + 1]);
        pack_ts_rect(mat.data(), C, Cn, tf, hp.data() + per * t);
      }
      uint4 *dr = nullptr, *dp = nullptr;
      if ((s = dev_alloc(h, h->arena, (void**)&dr, hr.size())) ||
          (s = dev_alloc(h, h->arena, (void**)&dp, hp.size())))
        return cleanup(), s;
      MCMG_CUDA(cudaMemcpyAsync(dr, hr.data(), hr.size(), cudaMemcpyHostToDevice, st));
      MCMG_CUDA(cudaMemcpyAsync(dp, hp.data(), hp.size(), cudaMemcpyHostToDevice, st));
      lv.ts_R = dr;
      lv.ts_P = dp;
      if (xts_block_pair(lv.g.d, Cn, C)) {
        // source s: rows [p C, (p + 1) C) hold P_o, o = p - 2 s per axis, for
        // every class p that reads s (s_a <= p_a), zeros for the others
        const int ncls = 1 << lv.g.d;
        const size_t perb = (tf ? 2 * sizeof(float) : sizeof(uint16_t)) * (size_t)(2 * Cn) *
                            (2 * C * ncls);
        std::vector<unsigned char> hb(perb * ncls);
        std::vector<float2> sm((size_t)ncls * C * Cn);
        for (int sv = 0; sv < ncls; ++sv) {
          for (int pc = 0; pc < ncls; ++pc) {
            int t = 0, mul = 1;
            bool used = true;
            for (int a = 0; a < lv.g.d; ++a, mul *= 3) {
              const int pa = (pc >> a) & 1, sa = (sv >> a) & 1;
              if (sa > pa) used = false;
              const int o = pa ? (sa ? -1 : 1) : 0;
              t += (o + 1) * mul;
            }
            const double* ps = lb[l].P + (size_t)2 * t * C * Cn;
            for (int cf = 0; cf < C; ++cf)
              for (int cc = 0; cc < Cn; ++cc) {
                const size_t i = (size_t)cf * Cn + cc;
                sm[((size_t)pc * C + cf) * Cn + cc] =
                    used ? make_float2((float)ps[2 * i], (float)ps[2 * i + 1]) : make_float2(0.f, 0.f);
              }
          }
          pack_ts_rect(sm.data(), ncls * C, Cn, tf, hb.data() + perb * sv);
        }
        uint4* db = nullptr;
        if ((s = dev_alloc(h, h->arena, (void**)&db, hb.size()))) return cleanup(), s;
        MCMG_CUDA(cudaMemcpyAsync(db, hb.data(), hb.size(), cudaMemcpyHostToDevice, st));
        lv.ts_Pb = db;
      }
    }
  }
  {
    std::vector<float2> vl(C0), vp(C0);
    for (int c2 = 0; c2 < C0; ++c2) {
      vl[c2] = make_float2((float)gl[2 * c2], (float)gl[2 * c2 + 1]);
      vp[c2] = make_float2((float)gp[2 * c2], (float)gp[2 * c2 + 1]);
    }
    if ((s = upload(h, h->arena, vl, &h->lift, st)) || (s = upload(h, h->arena, vp, &h->proj, st)))
      return cleanup(), s;
  }
  // ---- Algorithm 1 on the device
  float *m_in = nullptr, *net_a = nullptr, *net_s = nullptr, *net_n = nullptr;
  float *fw = nullptr, *fb = nullptr;
  if ((s = dev_alloc(h, tmp, (void**)&m_in, sizeof(float) * 2 * N))) return cleanup(), s;
  if ((s = launch_setup_input(h->q64, m_in, g0, st))) return cleanup(), s;
  {
    std::vector<float> wv = to_f32(flw, (size_t)2 * C0 * 2 * T3), bv = to_f32(flb, 2 * C0);
    if ((s = upload(h, tmp, wv, &fw, st)) || (s = upload(h, tmp, bv, &fb, st))) return cleanup(), s;
    if ((s = dev_alloc(h, tmp, (void**)&net_a, sizeof(float) * 2 * C0 * N))) return cleanup(), s;
    if ((s = launch_conv3_gelu(m_in, 2, net_a, 2 * C0, fw, fb, g0, 1, st))) return cleanup(), s;
  }
  double2* ql = h->q64;
  for (int l = 0; l < L; ++l) {
    Level& lv = h->lv[l];
    const int C = lv.C;
    const long long nl = lv.g.nodes();
    std::vector<float> sw = to_f32(lb[l].fsw, (size_t)2 * C * 2 * C * T3), sb = to_f32(lb[l].fsb, 2 * C);
    float *dsw, *dsb;
    if ((s = upload(h, tmp, sw, &dsw, st)) || (s = upload(h, tmp, sb, &dsb, st))) return cleanup(), s;
    if ((s = dev_alloc(h, tmp, (void**)&net_s, sizeof(float) * 2 * C * nl))) return cleanup(), s;
    if ((s = launch_conv3_gelu(net_a, 2 * C, net_s, 2 * C, dsw, dsb, lv.g, 1, st)))
      return cleanup(), s;
    if ((s = launch_assemble_features(net_a, net_s, ql, lv.a, lv.s, C, lv.g, l, w->feat_sl,
                                      w->feat_eps, w->sl_shift_re, w->sl_shift_im, st)))
      return cleanup(), s;
    if (l < L - 1) {
      const int Cn = lv.Cn;
      const Grid gc = lv.g.coarse();
      std::vector<float> aw = to_f32(lb[l].faw, (size_t)2 * Cn * 2 * C * T3), ab = to_f32(lb[l].fab, 2 * Cn);
      float *daw, *dab;
      if ((s = upload(h, tmp, aw, &daw, st)) || (s = upload(h, tmp, ab, &dab, st))) return cleanup(), s;
      if ((s = dev_alloc(h, tmp, (void**)&net_n, sizeof(float) * 2 * Cn * gc.nodes())))
        return cleanup(), s;
      if ((s = launch_conv3_gelu(net_a, 2 * C, net_n, 2 * Cn, daw, dab, lv.g, 2, st)))
        return cleanup(), s;
      double2* qn;
      if ((s = dev_alloc(h, tmp, (void**)&qn, sizeof(double2) * gc.nodes()))) return cleanup(), s;
      if ((s = launch_fw_restrict_q(ql, qn, lv.g, st))) return cleanup(), s;
      ql = qn;
      net_a = net_n;
    }
  }
  // autotune the CUDA-core smoothing shapes on scratch fields of the largest level
  {
    size_t big = 0;
    for (int l = 0; l < L; ++l)
      big = std::max(big, (size_t)h->lv[l].g.nodes() * h->lv[l].C);
    float2 *s0, *s1, *s2;
    if ((s = dev_alloc(h, tmp, (void**)&s0, sizeof(float2) * big)) ||
        (s = dev_alloc(h, tmp, (void**)&s1, sizeof(float2) * big)) ||
        (s = dev_alloc(h, tmp, (void**)&s2, sizeof(float2) * big)))
      return cleanup(), s;
    MCMG_CUDA(cudaMemsetAsync(s0, 0, sizeof(float2) * big, st));
    MCMG_CUDA(cudaMemsetAsync(s1, 0, sizeof(float2) * big, st));
    for (int l = 0; l < L; ++l) {
      if ((s = autotune_smooth(h->lv[l], s0, s1, s2, st))) return cleanup(), s;
      if (l < L - 1 && (s = autotune_transfer(h->lv[l], s0, s1, st))) return cleanup(), s;
    }
  }
  cudaError_t e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "setup");
  return MCMG_OK;
}

mcmg_status mcmg_setup(mcmg_ctx c, const mcmg_medium* m, double omega, const mcmg_weights* w,
                       mcmg_handle* out) {
  if (!c || !m || !w || !out || !m->c || !w->blob) {
    set_error("NULL argument");
    return MCMG_ERR_ARG;
  }
  if (m->dim != 2 && m->dim != 3) { set_error("dim must be 2 or 3"); return MCMG_ERR_ARG; }
  if (w->levels < 1 || w->levels > MCMG_MAX_LEVELS) {
    set_error("levels must be in 1..%d", MCMG_MAX_LEVELS);
    return MCMG_ERR_ARG;
  }
  if (w->precision != MCMG_FP32 && w->precision != MCMG_BF16 && w->precision != MCMG_FP32_TC) {
    set_error("unknown precision %d", w->precision);
    return MCMG_ERR_ARG;
  }
  for (int a = 0; a < m->dim; ++a)
    if (m->n[a] < 2) { set_error("grid axis %d too small", a); return MCMG_ERR_SHAPE; }
  {
    long long nodes = 1;
    for (int a = 0; a < m->dim; ++a) nodes *= m->n[a];
    if (nodes > 2147483647LL) {  // kernels index nodes in 32 bits
      set_error("grid of %lld nodes exceeds 2^31 - 1", nodes);
      return MCMG_ERR_SHAPE;
    }
  }
  MCMG_CUDA(cudaSetDevice(c->device));
  mcmg_handle_s* h = new mcmg_handle_s();
  h->ctx = c;
  h->device = c->device;
  cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaStreamCreate"); }
  e = cudaHostAlloc((void**)&h->err_host, sizeof(int), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&h->err_dev, h->err_host, 0);
  if (e != cudaSuccess) { mcmg_destroy(h); return cuda_fail(e, "error word"); }
  *h->err_host = 0;
  mcmg_status s = setup_impl(c, m, omega, w, h);
  if (s != MCMG_OK) {
    mcmg_destroy(h);
    return s;
  }
  *out = h;
  return MCMG_OK;
}

mcmg_status mcmg_destroy(mcmg_handle h) {
  if (!h) return MCMG_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->kry) krylov_destroy(h, h->kry);
  if (h->blk) block_destroy(h, h->blk);
  if (h->work) vwork_destroy(h, h->work);
  born_release(h);
  arena_free(h, h->arena);
  if (h->stream) cudaStreamDestroy(h->stream);
  if (h->err_host) cudaFreeHost(h->err_host);
  delete h;
  return MCMG_OK;
}

static mcmg_status ensure_work(mcmg_handle_s* h, int nrhs) {
  if (h->work && h->work->nrhs == nrhs) return MCMG_OK;
  if (h->work) {
    MCMG_CUDA(cudaDeviceSynchronize());
    vwork_destroy(h, h->work);
    h->work = nullptr;
  }
  return vwork_create(h, nrhs, &h->work);
}

mcmg_status mcmg_vcycle(mcmg_handle h, const void* r, void* e, int nrhs, void* stream) {
  if (!h || !r || !e || nrhs < 1) { set_error("bad argument"); return MCMG_ERR_ARG; }
  std::lock_guard<std::mutex> lk(h->mu);
  MCMG_CUDA(cudaSetDevice(h->device));
  MCMG_TRY(ensure_work(h, nrhs));
  return vcycle_run(h, h->work, (const float2*)r, (float2*)e, nrhs, (cudaStream_t)stream);
}

static mcmg_status check_opts(const mcmg_solve_opts* o) {
  if (!o || !(o->tol > 0.0) || o->restart_m < 1 || o->nrhs < 1 || o->max_iters < 0) {
    set_error("bad solve options");
    return MCMG_ERR_ARG;
  }
  return MCMG_OK;
}

// Order `work` after everything enqueued so far on the caller's stream
// (NULL: the legacy default stream), so that f and u written there before the
// call are what the solve reads.
static mcmg_status order_after(cudaStream_t caller, cudaStream_t work) {
  if (caller == work) return MCMG_OK;
  cudaEvent_t ev;
  MCMG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, caller);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(work, ev, 0);
  cudaEventDestroy(ev);
  if (e != cudaSuccess) return cuda_fail(e, "order after the caller's stream");
  return MCMG_OK;
}

mcmg_status mcmg_solve(mcmg_handle h, const void* f, void* u, const mcmg_solve_opts* o,
                       mcmg_solve_info* info) {
  if (!h || !f || !u) { set_error("NULL argument"); return MCMG_ERR_ARG; }
  MCMG_TRY(check_opts(o));
  std::lock_guard<std::mutex> lk(h->mu);
  MCMG_CUDA(cudaSetDevice(h->device));
  const bool plain_iter = (o->flags & (MCMG_SOLVE_STATIONARY | MCMG_SOLVE_BORN)) != 0;
  const int m_need = plain_iter ? 1 : o->restart_m;
  const bool batched = o->nrhs > 1 && !plain_iter;
  if (!batched) {
    if (h->kry && krylov_m(h->kry) != m_need) {
      krylov_destroy(h, h->kry);
      h->kry = nullptr;
    }
    if (!h->kry) MCMG_TRY(krylov_create(h, m_need, &h->kry));
  }
  const long long N = h->g0.nodes();
  mcmg_solve_info agg{};
  agg.converged = 1;
  mcmg_status worst = MCMG_OK;
  auto t0 = std::chrono::steady_clock::now();
  if (batched) {
    // all right-hand sides together: V-cycles batched per round
    if (h->blk && (block_m(h->blk) != o->restart_m || block_size(h->blk) != o->nrhs)) {
      block_destroy(h, h->blk);
      h->blk = nullptr;
    }
    if (!h->blk) MCMG_TRY(block_create(h, o->restart_m, o->nrhs, &h->blk));
    MCMG_TRY(order_after((cudaStream_t)o->stream, block_stream(h->blk)));
    MCMG_TRY(block_begin(h->blk, (const double2*)f, (double2*)u, *o));
    int done = 0;
    while (!done) MCMG_TRY(block_advance(h->blk, true, &done));
    block_info(h->blk, &agg, &worst);
  } else {
    if (!o->stream) MCMG_TRY(order_after(nullptr, h->stream));
    for (int k = 0; k < o->nrhs; ++k) {
      cudaStream_t st = o->stream ? (cudaStream_t)o->stream : h->stream;
      mcmg_solve_info one;
      mcmg_status fs;
      if (o->flags & MCMG_SOLVE_BORN) {
        MCMG_TRY(born_run(h->kry, (const double2*)f + (size_t)k * N,
                          (double2*)u + (size_t)k * N, *o, st, &one, &fs));
      } else if (o->flags & MCMG_SOLVE_STATIONARY) {
        MCMG_TRY(stationary_run(h->kry, (const double2*)f + (size_t)k * N,
                                (double2*)u + (size_t)k * N, *o, st, &one, &fs));
      } else {
        MCMG_TRY(krylov_begin(h->kry, (const double2*)f + (size_t)k * N,
                              (double2*)u + (size_t)k * N, *o, st));
        int done = 0;
        while (!done) MCMG_TRY(krylov_advance(h->kry, true, &done));
        krylov_info(h->kry, &one, &fs);
      }
      agg.iters = std::max(agg.iters, one.iters);
      agg.restarts = std::max(agg.restarts, one.restarts);
      agg.rel_residual = std::max(agg.rel_residual, one.rel_residual);
      agg.converged &= one.converged;
      if (fs != MCMG_OK && worst == MCMG_OK) worst = fs;
    }
  }
  agg.t_solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = agg;
  if (worst == MCMG_ERR_NOT_CONVERGED) set_error("max_iters reached above tolerance");
  return worst;
}

mcmg_status mcmg_solve_host(mcmg_handle h, const void* f_host, void* u_host,
                            const mcmg_solve_opts* o, mcmg_solve_info* info) {
  if (!h || !f_host || !u_host) { set_error("NULL argument"); return MCMG_ERR_ARG; }
  MCMG_TRY(check_opts(o));
  MCMG_CUDA(cudaSetDevice(h->device));
  const size_t bytes = sizeof(double2) * (size_t)h->g0.nodes() * o->nrhs;
  DevArena a;
  void *fd = nullptr, *ud = nullptr;
  mcmg_status s;
  if ((s = dev_alloc(h, a, &fd, bytes)) || (s = dev_alloc(h, a, &ud, bytes))) {
    arena_free(h, a);
    return s;
  }
  cudaError_t e = cudaMemcpyAsync(fd, f_host, bytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ud, u_host, bytes, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) { arena_free(h, a); return cuda_fail(e, "copy in"); }
  s = mcmg_solve(h, fd, ud, o, info);
  e = cudaMemcpyAsync(u_host, ud, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  arena_free(h, a);
  if (e != cudaSuccess) return cuda_fail(e, "copy out");
  return s;
}

// ---------------------------------------------------------- single steps ----
static mcmg_status check_level(mcmg_handle h, int level, bool need_next) {
  if (!h || level < 0 || level >= h->L || (need_next && level >= h->L - 1)) {
    set_error("level %d out of range", level);
    return MCMG_ERR_ARG;
  }
  return MCMG_OK;
}

int mcmg_kernel_shape_count(int op) { return op < 0 || op > 3 ? 0 : kernel_shape_count(op); }

mcmg_status mcmg_get_kernel_shape(mcmg_handle h, int level, int op, int* shape) {
  MCMG_TRY(check_level(h, level, op >= 2));
  if (!shape || op < 0 || op > 3) { set_error("bad argument"); return MCMG_ERR_ARG; }
  *shape = h->lv[level].shape[op];
  return MCMG_OK;
}

mcmg_status mcmg_set_kernel_shape(mcmg_handle h, int level, int op, int shape) {
  MCMG_TRY(check_level(h, level, op >= 2));
  if (op < 0 || op > 3 || shape < -1 || shape >= kernel_shape_count(op)) {
    set_error("bad argument");
    return MCMG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(h->mu);
  Level& lv = h->lv[level];
  if (shape >= 0 && !kernel_shape_valid(lv, op, shape)) {
    set_error("shape %d cannot run operation %d on level %d", shape, op, level);
    return MCMG_ERR_SHAPE;
  }
  const int want = shape < 0 ? lv.tuned[op] : shape;
  if (want != lv.shape[op]) {
    lv.shape[op] = want;
    ++h->shape_gen;
  }
  return MCMG_OK;
}

mcmg_status mcmg_device_error(mcmg_handle h, int* code) {
  if (!h || !code) { set_error("NULL argument"); return MCMG_ERR_ARG; }
  MCMG_CUDA(cudaSetDevice(h->device));
  MCMG_CUDA(cudaDeviceSynchronize());
  *code = *(volatile int*)h->err_host;
  return MCMG_OK;
}

mcmg_status mcmg_apply_A(mcmg_handle h, const void* x, void* y, int fp64, int nrhs, void* stream) {
  if (!h || !x || !y || nrhs < 1) { set_error("bad argument"); return MCMG_ERR_ARG; }
  MCMG_CUDA(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (fp64) return launch_apply_A64(h->q64, (const double2*)x, (double2*)y, h->g0, nrhs, st);
  return launch_apply_A32(h->q32, (const float2*)x, (float2*)y, h->g0, nrhs, st);
}

mcmg_status mcmg_get_feature(mcmg_handle h, int level, int which, void* out) {
  MCMG_TRY(check_level(h, level, false));
  if (!out || (which != 0 && which != 1)) { set_error("bad argument"); return MCMG_ERR_ARG; }
  const Level& lv = h->lv[level];
  MCMG_CUDA(cudaMemcpy(out, which == 0 ? lv.a : lv.s, sizeof(float2) * lv.g.nodes() * lv.C,
                       cudaMemcpyDeviceToDevice));
  return MCMG_OK;
}

mcmg_status mcmg_lift(mcmg_handle h, const void* r, void* r1, int nrhs, void* stream) {
  if (!h || !r || !r1 || nrhs < 1) { set_error("bad argument"); return MCMG_ERR_ARG; }
  return launch_lift((const float2*)r, h->lift, (float2*)r1, h->lv[0].C, h->g0.nodes(), nrhs,
                     (cudaStream_t)stream);
}

mcmg_status mcmg_project(mcmg_handle h, const void* e1, void* e, int nrhs, void* stream) {
  if (!h || !e1 || !e || nrhs < 1) { set_error("bad argument"); return MCMG_ERR_ARG; }
  return launch_project((const float2*)e1, h->proj, (float2*)e, h->lv[0].C, h->g0.nodes(), nrhs,
                        (cudaStream_t)stream);
}

mcmg_status mcmg_smooth(mcmg_handle h, int level, int step, const void* r, const void* e_in,
                        void* e_out, int nrhs, void* stream) {
  MCMG_TRY(check_level(h, level, false));
  const Level& lv = h->lv[level];
  if (!r || !e_out || nrhs < 1 || step < 0 || step >= lv.nu_pre + lv.nu_post) {
    set_error("bad argument");
    return MCMG_ERR_ARG;
  }
  return launch_smooth(lv, step, (const float2*)r, (const float2*)e_in, (float2*)e_out, 0, nrhs,
                       (cudaStream_t)stream);
}

mcmg_status mcmg_residual_restrict(mcmg_handle h, int level, const void* r, const void* e,
                                   void* rc, int nrhs, void* stream) {
  MCMG_TRY(check_level(h, level, true));
  if (!r || !e || !rc || nrhs < 1) { set_error("bad argument"); return MCMG_ERR_ARG; }
  std::lock_guard<std::mutex> lk(h->mu);
  MCMG_TRY(ensure_work(h, nrhs));
  const Level& lv = h->lv[level];
  cudaStream_t st = (cudaStream_t)stream;
  MCMG_TRY(launch_smooth(lv, 0, (const float2*)r, (const float2*)e, h->work->t[level], 1, nrhs, st));
  return launch_restrict(lv, h->work->t[level], (float2*)rc, nrhs, st);
}

mcmg_status mcmg_residual(mcmg_handle h, int level, const void* r, const void* e, void* t,
                          int nrhs, void* stream) {
  MCMG_TRY(check_level(h, level, false));
  if (!r || !e || !t || nrhs < 1 || t == e) { set_error("bad argument"); return MCMG_ERR_ARG; }
  return launch_smooth(h->lv[level], 0, (const float2*)r, (const float2*)e, (float2*)t, 1, nrhs,
                       (cudaStream_t)stream);
}

mcmg_status mcmg_coarse_basis(mcmg_handle h, int level, long long node, int channel, void* out,
                              void* stream) {
  if (!h || !out || level < 1 || level >= h->L || channel < 0 || channel >= h->lv[level].C ||
      node < 0 || node >= h->lv[level].g.nodes()) {
    set_error("bad argument");
    return MCMG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(h->mu);
  MCMG_CUDA(cudaSetDevice(h->device));
  MCMG_TRY(ensure_work(h, 1));
  cudaStream_t st = (cudaStream_t)stream;
  VWork* w = h->work;
  const Level& top = h->lv[level];
  // delta_alpha on `level`, then P_l for l = level-1 .. 0 into zeroed fields
  MCMG_CUDA(cudaMemsetAsync(w->e[level], 0, sizeof(float2) * top.g.nodes() * top.C, st));
  const float2 one = make_float2(1.f, 0.f);
  MCMG_CUDA(cudaMemcpyAsync(w->e[level] + node * top.C + channel, &one, sizeof(float2),
                            cudaMemcpyHostToDevice, st));
  for (int l = level - 1; l >= 0; --l) {
    const Level& lv = h->lv[l];
    MCMG_CUDA(cudaMemsetAsync(w->e[l], 0, sizeof(float2) * lv.g.nodes() * lv.C, st));
    MCMG_TRY(launch_prolong_add(lv, w->e[l + 1], w->e[l], 1, st));
  }
  const Level& l0 = h->lv[0];
  return launch_project(w->e[0], h->proj, (float2*)out, l0.C, l0.g.nodes(), 1, st);
}

mcmg_status mcmg_prolong_add(mcmg_handle h, int level, const void* ec, void* e, int nrhs,
                             void* stream) {
  MCMG_TRY(check_level(h, level, true));
  if (!ec || !e || nrhs < 1) { set_error("bad argument"); return MCMG_ERR_ARG; }
  return launch_prolong_add(h->lv[level], (const float2*)ec, (float2*)e, nrhs, (cudaStream_t)stream);
}

mcmg_status mcmg_cgs2(mcmg_handle h, const void* V, int k, size_t n, void* w, double* h_host,
                      double* norm_host) {
  if (!h || !V || !w || !h_host || !norm_host || k < 1 || n < 1) {
    set_error("bad argument");
    return MCMG_ERR_ARG;
  }
  MCMG_CUDA(cudaSetDevice(h->device));
  return cgs2_once(h, (const float2*)V, k, (long long)n, (float2*)w, h_host, norm_host, h->stream);
}

// ------------------------------------------------------------------ server --
// One worker thread.  Admission: queued requests start in arrival order when
// their Krylov and V-cycle workspaces fit the context's HBM budget.  Each
// admitted request runs as one block solve on its own stream: per round, the
// V-cycles of all its right-hand sides that need one run as a single batched
// launch per level.  The worker polls every request's last event and enqueues
// its next round as soon as it completes, so different requests overlap on the
// device.

static size_t request_bytes(mcmg_handle_s* h, const mcmg_solve_opts& o) {
  const size_t n = (size_t)h->g0.nodes();
  const int m = o.restart_m;
  size_t b = sizeof(float2) * n * (2 * (size_t)m + 2) + sizeof(double2) * n;
  for (int l = 0; l < h->L; ++l) b += 4 * sizeof(float2) * (size_t)h->lv[l].g.nodes() * h->lv[l].C;
  b += sizeof(double2) * (size_t)m * (m + 1) + ((size_t)1 << 20);
  return b * o.nrhs;
}

static void release(Request* r) {
  if (r->blk) {
    block_destroy(r->h, r->blk);
    r->blk = nullptr;
  }
}

static bool try_admit(mcmg_ctx_s* c, Request* r) {
  if (c->budget && c->used.load() + r->bytes_needed > c->budget) {
    set_error("request needs about %zu bytes; %zu of the %zu-byte budget are in use",
              r->bytes_needed, c->used.load(), c->budget);
    r->err = mcmg_last_error();
    return false;
  }
  mcmg_status s = block_create(r->h, r->o.restart_m, r->o.nrhs, &r->blk);
  if (s != MCMG_OK) {
    r->err = mcmg_last_error();
    release(r);
    cudaGetLastError();
    return false;
  }
  // the request reads f and u only after the caller's work before the submit
  if (r->ready) {
    cudaError_t e = cudaStreamWaitEvent(block_stream(r->blk), r->ready, 0);
    cudaEventDestroy(r->ready);
    r->ready = nullptr;
    if (e != cudaSuccess) {
      r->status = cuda_fail(e, "wait for the caller's stream");
      r->err = mcmg_last_error();
      return true;
    }
  }
  s = block_begin(r->blk, r->f, r->u, r->o);
  if (s != MCMG_OK) {
    r->status = s;
    r->err = mcmg_last_error();
  }
  return true;
}

// ---- cross-request batching --------------------------------------------
// One V-cycle (Algorithm 2) for the pending right-hand sides of several
// requests whose handles share weights and level layout (wsig), each with its
// own medium (features) and grid.  Per level, every smoothing step and the
// residual of all members is one tensor-core launch over all their fields
// (field descriptors: pointers, features, grid); lift, restriction,
// prolongation and projection run per member.  Every field goes through the
// same arithmetic as in a V-cycle of its own, so results are unchanged by the
// company a request keeps.  The launches run on the server's stream, ordered
// after each member's stream and back.
struct CohortMember {
  mcmg_handle_s* h;
  VWork* w;
  const float2* const* srcs;
  float2* const* dsts;
  int count;
  cudaStream_t st;
  float2* ecur[MCMG_MAX_LEVELS];
};

namespace {

struct CohortOp {
  enum Kind { TS, SMOOTH, RESTRICT, PROLONG, MEMSET } kind;
  int member = -1, level = 0, step = 0, mode = 0;
  int f0 = 0, nf = 0;                 // TS: descriptors [f0, f0 + nf)
  bool has_e = false;
  const float2* r = nullptr;          // SMOOTH (one member, CUDA cores)
  const float2* e_in = nullptr;
  float2* out = nullptr;
};

}  // namespace

static mcmg_status cohort_vcycle(mcmg_ctx_s* c, std::vector<CohortMember>& ms, bool* planned) {
  *planned = false;
  // ---- plan: the level sequence of every member, batched per level
  std::vector<CohortOp> ops;
  std::vector<TsField> fd;
  int Lmax = 0;
  for (auto& m : ms) Lmax = std::max(Lmax, m.h->L);
  auto fields_of = [&](int l, const std::vector<int>& who, const float2* const* eins,
                       float2* const* outs, bool use_t_out) {
    // one descriptor per (member, right-hand side)
    const int f0 = (int)fd.size();
    int first = 0;
    for (size_t q = 0; q < who.size(); ++q) {
      const CohortMember& m = ms[who[q]];
      const Level& lv = m.h->lv[l];
      const long long nl = lv.g.nodes();
      const size_t stride = (size_t)nl * lv.C;
      for (int k = 0; k < m.count; ++k) {
        TsField f{};
        f.r = m.w->r[l] + k * stride;
        f.e_in = eins[q] ? eins[q] + k * stride : nullptr;
        f.out = (use_t_out ? m.w->t[l] : outs[q]) + k * stride;
        f.a = lv.a;
        f.s = lv.s;
        f.nodes = nl;
        f.nx = lv.g.nx;
        f.ny = lv.g.ny;
        f.nz = lv.g.nz;
        f.tiles = (int)((nl + 127) / 128);
        f.first = first;
        first += f.tiles;
        fd.push_back(f);
      }
    }
    return std::make_pair(f0, (int)fd.size() - f0);
  };
  bool same = true;                   // every batched launch's arithmetic agrees
  auto steps = [&](int l, const std::vector<int>& who, int step0, int nsteps, bool from_zero) {
    const Level& L0 = ms[who[0]].h->lv[l];
    for (int q : who)
      for (int i = 0; i < nsteps; ++i)
        if (step0 + i > 2 * 8 || ms[q].h->lv[l].ssig[step0 + i] != L0.ssig[step0 + i] ||
            ms[q].h->lv[l].use_ts != L0.use_ts)
          same = false;
    for (int i = 0; i < nsteps; ++i) {
      std::vector<const float2*> eins(who.size());
      std::vector<float2*> outs(who.size());
      for (size_t q = 0; q < who.size(); ++q) {
        CohortMember& m = ms[who[q]];
        float2* cur = (from_zero && i == 0) ? nullptr : m.ecur[l];
        eins[q] = cur;
        outs[q] = (cur == m.w->e[l]) ? m.w->e2[l] : m.w->e[l];
      }
      if (L0.use_ts) {
        auto fr = fields_of(l, who, eins.data(), outs.data(), false);
        CohortOp op{CohortOp::TS};
        op.level = l;
        op.step = step0 + i;
        op.mode = 0;
        op.f0 = fr.first;
        op.nf = fr.second;
        op.has_e = eins[0] != nullptr;
        op.member = who[0];
        ops.push_back(op);
      } else {
        for (size_t q = 0; q < who.size(); ++q) {
          CohortOp op{CohortOp::SMOOTH};
          op.member = who[q];
          op.level = l;
          op.step = step0 + i;
          op.mode = 0;
          op.r = ms[who[q]].w->r[l];
          op.e_in = eins[q];
          op.out = outs[q];
          ops.push_back(op);
        }
      }
      for (size_t q = 0; q < who.size(); ++q) ms[who[q]].ecur[l] = outs[q];
    }
  };
  for (int l = 0; l < Lmax; ++l) {                   // down cycle
    std::vector<int> who, res;
    for (int q = 0; q < (int)ms.size(); ++q)
      if (ms[q].h->L > l) who.push_back(q);
    const int nu = ms[who[0]].h->lv[l].nu_pre;
    for (int q : who)
      if (ms[q].h->lv[l].nu_pre != nu) return MCMG_OK;   // not batchable: caller runs them apart
    if (nu > 0) {
      steps(l, who, 0, nu, true);
    } else {
      for (int q : who) {
        CohortOp op{CohortOp::MEMSET};
        op.member = q;
        op.level = l;
        ops.push_back(op);
        ms[q].ecur[l] = ms[q].w->e[l];
      }
    }
    for (int q : who)
      if (l < ms[q].h->L - 1) res.push_back(q);
    if (!res.empty()) {
      const Level& L0 = ms[res[0]].h->lv[l];
      for (int q : res)
        if (ms[q].h->lv[l].rsig != L0.rsig || ms[q].h->lv[l].use_ts != L0.use_ts) same = false;
      std::vector<const float2*> eins(res.size());
      for (size_t q = 0; q < res.size(); ++q) eins[q] = ms[res[q]].ecur[l];
      if (L0.use_ts) {
        auto fr = fields_of(l, res, eins.data(), nullptr, true);
        CohortOp op{CohortOp::TS};
        op.level = l;
        op.mode = 1;
        op.f0 = fr.first;
        op.nf = fr.second;
        op.has_e = true;
        op.member = res[0];
        ops.push_back(op);
      } else {
        for (size_t q = 0; q < res.size(); ++q) {
          CohortOp op{CohortOp::SMOOTH};
          op.member = res[q];
          op.level = l;
          op.mode = 1;
          op.r = ms[res[q]].w->r[l];
          op.e_in = eins[q];
          op.out = ms[res[q]].w->t[l];
          ops.push_back(op);
        }
      }
      for (int q : res) {
        CohortOp op{CohortOp::RESTRICT};
        op.member = q;
        op.level = l;
        ops.push_back(op);
      }
    }
  }
  for (int l = Lmax - 2; l >= 0; --l) {              // up cycle
    std::vector<int> who;
    for (int q = 0; q < (int)ms.size(); ++q)
      if (l < ms[q].h->L - 1) who.push_back(q);
    if (who.empty()) continue;
    const int nu = ms[who[0]].h->lv[l].nu_post, nu1 = ms[who[0]].h->lv[l].nu_pre;
    for (int q : who)
      if (ms[q].h->lv[l].nu_post != nu || ms[q].h->lv[l].nu_pre != nu1) return MCMG_OK;
    for (int q : who) {
      CohortOp op{CohortOp::PROLONG};
      op.member = q;
      op.level = l;
      op.e_in = ms[q].ecur[l + 1];      // the pointers as they are at this point of the cycle
      op.out = ms[q].ecur[l];
      ops.push_back(op);
    }
    if (nu > 0) steps(l, who, nu1, nu, false);
  }
  if (!same || (int)fd.size() > c->fd_cap) return MCMG_OK;   // run the members apart
  *planned = true;

  // ---- lift on each member's stream; the server stream follows all of them
  for (auto& m : ms) {
    const Level& l0 = m.h->lv[0];
    MCMG_TRY(launch_lift_gather(m.srcs, m.h->lift, m.w->r[0], l0.C, l0.g.nodes(), m.count, m.st));
    MCMG_TRY(order_after(m.st, c->sst));
  }
  // ---- descriptors: one upload (the staging is rewritten only once the
  // previous upload has been read)
  if (!fd.empty()) {
    MCMG_CUDA(cudaEventSynchronize(c->fd_ev));
    std::memcpy(c->fd_h, fd.data(), sizeof(TsField) * fd.size());
    MCMG_CUDA(cudaMemcpyAsync(c->fd_d, c->fd_h, sizeof(TsField) * fd.size(),
                              cudaMemcpyHostToDevice, c->sst));
    MCMG_CUDA(cudaEventRecord(c->fd_ev, c->sst));
  }
  for (const CohortOp& op : ops) {
    CohortMember& m = ms[op.member];
    const Level& lv = m.h->lv[op.level];
    switch (op.kind) {
      case CohortOp::TS:
        MCMG_TRY(launch_smooth_ts_fields(lv, op.step, c->fd_d + op.f0, fd.data() + op.f0, op.nf,
                                         op.has_e, op.mode, c->sst));
        break;
      case CohortOp::SMOOTH:
        MCMG_TRY(launch_smooth(lv, op.step, op.r, op.e_in, op.out, op.mode, m.count, c->sst));
        break;
      case CohortOp::RESTRICT:
        MCMG_TRY(launch_restrict(lv, m.w->t[op.level], m.w->r[op.level + 1], m.count, c->sst));
        break;
      case CohortOp::PROLONG:
        MCMG_TRY(launch_prolong_add(lv, op.e_in, op.out, m.count, c->sst));
        break;
      case CohortOp::MEMSET:
        MCMG_CUDA(cudaMemsetAsync(m.w->e[op.level], 0,
                                  sizeof(float2) * lv.g.nodes() * lv.C * m.count, c->sst));
        break;
    }
  }
  // ---- projection on each member's stream, after the server stream
  for (auto& m : ms) {
    const Level& l0 = m.h->lv[0];
    MCMG_TRY(order_after(c->sst, m.st));
    MCMG_TRY(launch_project_scatter(m.ecur[0], m.h->proj, m.dsts, l0.C, l0.g.nodes(), m.count,
                                    m.st));
  }
  c->cohort_rounds += 1;
  c->cohort_members += ms.size();
  return MCMG_OK;
}

// The server thread's stream and descriptor staging, made on first use.
static mcmg_status server_resources(mcmg_ctx_s* c) {
  if (c->sst) return MCMG_OK;
  const int cap = 16384;
  MCMG_CUDA(cudaStreamCreateWithFlags(&c->sst, cudaStreamNonBlocking));
  MCMG_CUDA(cudaEventCreateWithFlags(&c->fd_ev, cudaEventDisableTiming));
  MCMG_CUDA(cudaHostAlloc((void**)&c->fd_h, sizeof(TsField) * cap, cudaHostAllocDefault));
  MCMG_CUDA(cudaMalloc((void**)&c->fd_d, sizeof(TsField) * cap));
  c->fd_cap = cap;
  return MCMG_OK;
}

static void server_loop(mcmg_ctx_s* c) {
  cudaSetDevice(c->device);
  std::unique_lock<std::mutex> lk(c->mu);
  while (!c->stop) {
    // admit in arrival order
    while (!c->queue.empty()) {
      Request* r = c->queue.front();
      if (!try_admit(c, r)) {
        if (c->active.empty()) {   // can never fit: fail it
          r->status = MCMG_ERR_OOM;
          c->queue.pop_front();
          c->finished[r->ticket] = r;
          continue;
        }
        break;
      }
      c->queue.pop_front();
      c->active.push_back(r);
    }
    if (c->active.empty()) {
      c->cv.notify_all();
      c->cv.wait(lk, [&] { return c->stop || !c->queue.empty(); });
      continue;
    }
    const bool batch = c->batching;
    lk.unlock();
    bool progressed = false;
    std::vector<Request*> fin, ready;
    std::vector<int> counts;
    for (Request* r : c->active) {
      bool all = r->status != MCMG_PENDING;
      if (!all) {
        int d = 0, cnt = -1;
        mcmg_status s = block_poll(r->blk, false, &d, &cnt);
        if (s != MCMG_OK) { r->status = s; r->err = mcmg_last_error(); d = 1; }
        if (d) {
          all = true;
          progressed = true;
        } else if (cnt >= 0) {                 // its round finished: a new one starts now
          ready.push_back(r);
          counts.push_back(cnt);
          progressed = true;
        }
      }
      if (all) fin.push_back(r);
    }
    // the V-cycles of this round: requests that share weights and level
    // layout run as one cohort (one launch per level and step for all of
    // them), the others each on its own stream
    if (!ready.empty()) {
      std::map<uint64_t, std::vector<int>> groups;
      for (int i = 0; i < (int)ready.size(); ++i)
        if (counts[i] > 0) groups[batch ? ready[i]->h->wsig : (uint64_t)i].push_back(i);
      for (auto& g : groups) {
        bool done_g = false;
        if (g.second.size() >= 2 && server_resources(c) == MCMG_OK) {
          std::vector<CohortMember> ms;
          for (int i : g.second) {
            CohortMember m{};
            m.h = ready[i]->h;
            block_vcycle_io(ready[i]->blk, &m.w, &m.srcs, &m.dsts);
            m.count = counts[i];
            m.st = block_stream(ready[i]->blk);
            ms.push_back(m);
          }
          bool planned = false;
          mcmg_status s = cohort_vcycle(c, ms, &planned);
          if (s != MCMG_OK) {
            for (int i : g.second) { ready[i]->status = s; ready[i]->err = mcmg_last_error(); }
            planned = true;
          }
          done_g = planned;
        }
        if (!done_g) {
          for (int i : g.second) {
            VWork* w;
            const float2* const* srcs;
            float2* const* dsts;
            block_vcycle_io(ready[i]->blk, &w, &srcs, &dsts);
            mcmg_status s = vcycle_run_batch(ready[i]->h, w, srcs, dsts, counts[i],
                                             block_stream(ready[i]->blk));
            if (s != MCMG_OK) { ready[i]->status = s; ready[i]->err = mcmg_last_error(); }
          }
        }
      }
      for (Request* r : ready) {
        if (r->status != MCMG_PENDING) continue;
        mcmg_status s = block_after_vcycle(r->blk);
        if (s != MCMG_OK) { r->status = s; r->err = mcmg_last_error(); }
      }
    }
    for (Request* r : fin) {
      mcmg_solve_info agg{};
      mcmg_status worst = r->status == MCMG_PENDING ? MCMG_OK : r->status;
      if (r->blk) {
        mcmg_status fs;
        block_info(r->blk, &agg, &fs);
        if (fs != MCMG_OK && worst == MCMG_OK) worst = fs;
      }
      agg.t_solve_s =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - r->t_submit).count();
      r->info = agg;
      r->status = worst;
      release(r);
    }
    lk.lock();
    for (Request* r : fin) {
      c->active.erase(std::find(c->active.begin(), c->active.end(), r));
      c->finished[r->ticket] = r;
    }
    if (!fin.empty()) c->cv.notify_all();
    if (!progressed && fin.empty()) {
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    }
  }
}

static void server_start(mcmg_ctx_s* c) {
  if (c->running) return;
  c->stop = false;
  c->running = true;
  c->worker = std::thread(server_loop, c);
}

static void server_stop(mcmg_ctx_s* c) {
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->running) return;
    c->stop = true;
  }
  c->cv.notify_all();
  c->worker.join();
  c->running = false;
  for (Request* r : c->active) { release(r); delete r; }
  for (Request* r : c->queue) delete r;
  c->active.clear();
  c->queue.clear();
  cudaSetDevice(c->device);
  if (c->sst) {
    cudaStreamSynchronize(c->sst);
    cudaStreamDestroy(c->sst);
    c->sst = nullptr;
  }
  if (c->fd_ev) { cudaEventDestroy(c->fd_ev); c->fd_ev = nullptr; }
  if (c->fd_h) { cudaFreeHost(c->fd_h); c->fd_h = nullptr; }
  if (c->fd_d) { cudaFree(c->fd_d); c->fd_d = nullptr; }
  c->fd_cap = 0;
}

mcmg_status mcmg_submit(mcmg_ctx c, mcmg_handle h, const void* f, void* u,
                        const mcmg_solve_opts* o, uint64_t* ticket) {
  if (!c || !h || !f || !u || !ticket || h->ctx != c) {
    set_error("bad argument");
    return MCMG_ERR_ARG;
  }
  MCMG_TRY(check_opts(o));
  if (o->flags & (MCMG_SOLVE_STATIONARY | MCMG_SOLVE_BORN)) {
    set_error("the server runs FGMRES solves only (no stationary or Born iteration)");
    return MCMG_ERR_ARG;
  }
  Request* r = new Request();
  r->h = h;
  r->f = (const double2*)f;
  r->u = (double2*)u;
  r->o = *o;
  {
    // mark the caller's stream now; the server orders the request after it
    cudaError_t e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r->ready, (cudaStream_t)o->stream);
    if (e != cudaSuccess) {
      if (r->ready) cudaEventDestroy(r->ready);
      delete r;
      return cuda_fail(e, "record the caller's stream");
    }
  }
  r->bytes_needed = request_bytes(h, *o);
  r->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->queue.size() >= c->max_queue) {
      delete r;
      set_error("server queue full");
      return MCMG_ERR_BUSY;
    }
    r->ticket = c->next_ticket++;
    c->queue.push_back(r);
    *ticket = r->ticket;
    server_start(c);
  }
  c->cv.notify_all();
  return MCMG_OK;
}

mcmg_status mcmg_server_batching(mcmg_ctx c, int enable, uint64_t* rounds, uint64_t* members) {
  if (!c) { set_error("NULL context"); return MCMG_ERR_ARG; }
  std::lock_guard<std::mutex> lk(c->mu);
  if (enable >= 0) c->batching = enable != 0;
  if (rounds) *rounds = c->cohort_rounds;
  if (members) *members = c->cohort_members;
  return MCMG_OK;
}

mcmg_status mcmg_poll(mcmg_ctx c, uint64_t ticket, mcmg_solve_info* info) {
  if (!c) { set_error("NULL context"); return MCMG_ERR_ARG; }
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->finished.find(ticket);
  if (it == c->finished.end()) {
    for (Request* r : c->queue)
      if (r->ticket == ticket) return MCMG_PENDING;
    for (Request* r : c->active)
      if (r->ticket == ticket) return MCMG_PENDING;
    set_error("unknown ticket %llu", (unsigned long long)ticket);
    return MCMG_ERR_ARG;
  }
  Request* r = it->second;
  if (info) *info = r->info;
  mcmg_status s = r->status;
  if (s < 0) set_error("%s", r->err.empty() ? "request failed" : r->err.c_str());
  c->finished.erase(it);
  delete r;
  return s;
}

mcmg_status mcmg_drain(mcmg_ctx c) {
  if (!c) { set_error("NULL context"); return MCMG_ERR_ARG; }
  std::unique_lock<std::mutex> lk(c->mu);
  c->cv.wait(lk, [&] { return c->queue.empty() && c->active.empty(); });
  return MCMG_OK;
}
