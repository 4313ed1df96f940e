// Request server: continuous batching of independent LocalPower solves.
//
// A request is one truncated-SVD problem (its partitions and its schedule).
// Requests wait in arrival order; lp_server_progress admits the head of the
// queue while the sum of the admitted requests' device-memory estimates stays
// within the budget and fewer than max_active are on the device.  An admitted
// request gets its own context (own stream, own device buffers): its partitions
// are copied in and its whole solve is enqueued at once, so A_i and the
// iterates stay resident across its rounds and the GPU interleaves its kernels
// with those of every other admitted request.  Completion is detected with the
// event the solve records last; the results move to host memory and the
// context is destroyed, which returns its budget share to the queue.
#include <cuda_runtime.h>

#include <algorithm>
#include <deque>
#include <new>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "lp_internal.cuh"

namespace {

struct Request {
  int64_t id = 0;
  // copies of the request's small arrays
  int m = 0;
  int64_t d = 0, pitch = 0;
  lp_dtype dtype = LP_F32;
  lp_ptr_space space = LP_HOST;
  std::vector<int64_t> rows;
  std::vector<const void*> parts;
  std::vector<const float*> scales;
  int k = 0, refine = 0, T = 0;
  lp_aggregator agg = LP_AGG_SIGN;
  unsigned flags = 0;
  std::vector<int> sched;
  std::vector<double> y0;
  size_t est = 0;
  // device side while active
  lp_ctx* ctx = nullptr;
  // results
  bool done = false;
  lp_status status = LP_OK;
  std::string err;
  std::vector<double> z, sigma;
  lp_stats stats{};
};

}  // namespace

struct lp_server {
  int device = 0;
  int sms = 0;
  size_t budget = 0;
  int max_active = 1;
  size_t in_use = 0, peak = 0;
  int64_t next_id = 1;
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::vector<int64_t> finished;  // completed since the last progress call
  std::unordered_map<int64_t, std::unique_ptr<Request>> all;
  std::string err;
};

namespace {

lp_status sfail(lp_server* s, lp_status st, const std::string& msg) {
  s->err = msg;
  return st;
}

void finish(lp_server* s, Request* r, lp_status st, const std::string& msg) {
  r->status = st;
  r->err = msg;
  r->done = true;
  s->finished.push_back(r->id);
}

void release(lp_server* s, Request* r) {
  if (r->ctx) {
    lp_destroy(r->ctx);
    r->ctx = nullptr;
    s->in_use -= r->est;
  }
}

// Copies the partitions in and enqueues the solve; failures complete the request.
void admit(lp_server* s, Request* r) {
  lp_ctx* c = nullptr;
  lp_status st = lp_create(&c, s->device, r->est, nullptr);
  if (st) {
    finish(s, r, st, lp_last_error(nullptr));
    return;
  }
  r->ctx = c;
  s->in_use += r->est;
  s->peak = std::max(s->peak, s->in_use);
  st = lp::load_pitched(c, r->m, r->rows.data(), r->d, r->pitch, r->dtype, r->parts.data(),
                        r->dtype == LP_FP8_E4M3 ? r->scales.data() : nullptr, r->space);
  if (!st)
    st = lp_solve(c, r->k, r->sched.empty() ? nullptr : r->sched.data(), r->T, r->agg, r->y0.data(), r->refine,
                  r->flags);
  if (st) {
    const std::string msg = lp_last_error(c);
    release(s, r);
    finish(s, r, st, msg);
    return;
  }
  s->active.push_back(r);
}

}  // namespace

extern "C" {

lp_status lp_server_create(lp_server** out, int device, size_t hbm_budget_bytes, int max_active) {
  if (!out) return LP_ERR_INVALID;
  *out = nullptr;
  if (max_active < 1) return LP_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    (void)cudaGetLastError();
    return ndev == 0 ? LP_ERR_CUDA : LP_ERR_INVALID;
  }
  lp_server* s = new (std::nothrow) lp_server();
  if (!s) return LP_ERR_OOM;
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  if (cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete s;
    return LP_ERR_CUDA;
  }
  *out = s;
  return LP_OK;
}

lp_status lp_server_submit(lp_server* s, const lp_request* q, int64_t* id) {
  if (!s) return LP_ERR_INVALID;
  s->err.clear();
  if (!q || !id) return sfail(s, LP_ERR_INVALID, "request and id must be non-NULL");
  *id = 0;
  if (q->m < 1 || !q->rows || !q->parts || q->d < 1 || q->k < 1 || q->k > LP_MAX_K || q->k > q->d || !q->y0 ||
      q->T < 0 || q->refine_rounds < 0 || q->T + q->refine_rounds < 1 || (q->T > 0 && !q->p_schedule))
    return sfail(s, LP_ERR_INVALID, "malformed request");
  if (q->row_pitch != 0 && q->row_pitch < q->d) return sfail(s, LP_ERR_INVALID, "row_pitch below d");
  if (q->dtype == LP_FP8_E4M3 && !q->row_scales) return sfail(s, LP_ERR_INVALID, "FP8 request needs row_scales");
  for (int i = 0; i < q->m; ++i) {
    if (q->rows[i] < q->k) return sfail(s, LP_ERR_INVALID, "k exceeds a partition's row count");
    if (!q->parts[i]) return sfail(s, LP_ERR_INVALID, "NULL partition pointer");
  }
  for (int t = 0; t < q->T; ++t)
    if (q->p_schedule[t] < 1) return sfail(s, LP_ERR_INVALID, "p_schedule entries must be >= 1");
  auto r = std::make_unique<Request>();
  r->m = q->m;
  r->d = q->d;
  r->pitch = q->row_pitch ? q->row_pitch : q->d;
  r->dtype = q->dtype;
  r->space = q->space;
  r->rows.assign(q->rows, q->rows + q->m);
  r->parts.assign(q->parts, q->parts + q->m);
  if (q->dtype == LP_FP8_E4M3) r->scales.assign(q->row_scales, q->row_scales + q->m);
  r->k = q->k;
  r->T = q->T;
  r->refine = q->refine_rounds;
  r->agg = q->agg;
  r->flags = q->flags;
  if (q->T > 0) r->sched.assign(q->p_schedule, q->p_schedule + q->T);
  r->y0.assign(q->y0, q->y0 + size_t(q->d) * q->k);
  r->est = lp::estimate_bytes(s->sms, r->m, r->rows.data(), r->d, r->pitch, r->dtype, r->k, r->space);
  if (s->budget && r->est > s->budget)
    return sfail(s, LP_ERR_OOM, "request needs about " + std::to_string(r->est) + " bytes, over the server budget");
  r->id = s->next_id++;
  *id = r->id;
  s->queue.push_back(r.get());
  s->all.emplace(r->id, std::move(r));
  return LP_OK;
}

lp_status lp_server_progress(lp_server* s, int64_t* done_ids, int cap, int* n_done) {
  if (!s) return LP_ERR_INVALID;
  s->err.clear();
  if (n_done) *n_done = 0;
  if (cudaSetDevice(s->device) != cudaSuccess) {
    (void)cudaGetLastError();
    return sfail(s, LP_ERR_CUDA, "cudaSetDevice failed");
  }
  // retire
  for (size_t i = 0; i < s->active.size();) {
    Request* r = s->active[i];
    const int state = lp::solve_state(r->ctx);
    if (state == 0) {
      ++i;
      continue;
    }
    r->z.assign(size_t(r->d) * r->k, 0.0);
    r->sigma.assign(size_t(r->k), 0.0);
    const lp_status st = lp_result(r->ctx, r->z.data(), r->sigma.data(), &r->stats);
    const std::string msg = st ? lp_last_error(r->ctx) : "";
    release(s, r);
    finish(s, r, st, msg);
    s->active[i] = s->active.back();
    s->active.pop_back();
  }
  // admit in arrival order
  while (!s->queue.empty() && static_cast<int>(s->active.size()) < s->max_active) {
    Request* r = s->queue.front();
    if (s->budget && s->in_use + r->est > s->budget) break;
    s->queue.pop_front();
    admit(s, r);
  }
  // report
  int n = 0;
  while (n < cap && !s->finished.empty()) {
    if (done_ids) done_ids[n] = s->finished.front();
    s->finished.erase(s->finished.begin());
    ++n;
  }
  if (n_done) *n_done = n;
  return LP_OK;
}

lp_status lp_server_result(lp_server* s, int64_t id, double* z_out, double* sigma_out, lp_stats* stats) {
  if (!s) return LP_ERR_INVALID;
  s->err.clear();
  auto it = s->all.find(id);
  if (it == s->all.end() || !it->second->done) return sfail(s, LP_ERR_STATE, "request unknown or not complete");
  Request* r = it->second.get();
  const lp_status st = r->status;
  s->err = r->err;
  if (!st) {
    if (z_out) std::copy(r->z.begin(), r->z.end(), z_out);
    if (sigma_out) std::copy(r->sigma.begin(), r->sigma.end(), sigma_out);
  }
  if (stats) *stats = r->stats;
  s->finished.erase(std::remove(s->finished.begin(), s->finished.end(), id), s->finished.end());
  s->all.erase(it);
  return st;
}

lp_status lp_server_query(lp_server* s, lp_server_info* info) {
  if (!s || !info) return LP_ERR_INVALID;
  int64_t completed = 0;
  for (const auto& kv : s->all) completed += kv.second->done ? 1 : 0;
  info->queued = static_cast<int64_t>(s->queue.size());
  info->active = static_cast<int64_t>(s->active.size());
  info->completed = completed;
  info->hbm_in_use = s->in_use;
  info->hbm_peak = s->peak;
  info->hbm_budget = s->budget;
  return LP_OK;
}

const char* lp_server_error(const lp_server* s) { return s ? s->err.c_str() : ""; }

void lp_server_destroy(lp_server* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  for (Request* r : s->active) release(s, r);  // lp_destroy synchronises the request's stream
  delete s;
}

}  // extern "C"

// =============================================================================
// Batch runner: many independent instances solved by one CUDA graph launch.
//
// Each added instance is loaded into a context of its own (validation, packing,
// its copy of the data).  Before the first solve, instances that share the
// shape of the work - width d, storage type, k, schedule, aggregator and flags -
// are merged into one group context: their partitions are copied back to back
// into the group's buffers and each instance becomes one problem of the group
// (its own start block, bases, weights, aggregate and result).  A group's solve
// is then the ordinary launch sequence with every step kind covering all of the
// group's instances at once: one persistent step-kernel launch walks the row
// pieces of every partition of every instance (its work list, dealt to the
// CTAs by rows), one reduction, one batched CholQR2 over all partitions, one
// alignment, one aggregation and one batched CholQR2 over the problems.  The
// groups' sequences are captured into one graph as independent branches (a
// fork event on the batch stream, each group on its own stream, a join back),
// so the GPU runs different groups' kernels side by side; later solves replay
// the graph with one launch.  Each group's step kernel and tuning come from the
// autotuner, timed on the group's own data.
namespace {

struct Inst {
  Request q;            // parameters (q.ctx holds this instance's loaded data)
  int group = -1;       // group index
  int problem = -1;     // problem index inside the group
};

struct Group {
  lp_ctx* ctx = nullptr;
  std::vector<int> members;  // instance indices, in problem order
  std::vector<double> y0;    // members' start blocks back to back
  lp_stats captured{};
  cudaEvent_t join = nullptr, ready = nullptr;
};

// Instances of one group share every parameter of the launch sequence.
bool same_group(const Request& a, const Request& b) {
  return a.d == b.d && a.dtype == b.dtype && a.k == b.k && a.T == b.T && a.refine == b.refine && a.agg == b.agg &&
         a.flags == b.flags && a.sched == b.sched;
}

}  // namespace

struct lp_batch {
  int device = 0;
  int sms = 0;
  size_t budget = 0, in_use = 0;
  cudaStream_t root = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<std::unique_ptr<Inst>> inst;
  std::vector<std::unique_ptr<Group>> groups;
  bool grouped = false;   // groups reflect the current instances
  bool tuned = false;     // lp_batch_autotune asked for tuned groups
  cudaGraphExec_t exec = nullptr;
  bool solved = false;
  std::string err;
};

namespace {

lp_status bfail(lp_batch* b, lp_status st, const std::string& msg) {
  b->err = msg;
  return st;
}

void drop_batch_graph(lp_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->solved = false;
}

// The group contexts go only after a batch solve still running on the root
// stream (a later add or autotune may follow a solve without a result call).
void drop_groups(lp_batch* b) {
  if (b->root && (b->exec || !b->groups.empty()) && cudaStreamSynchronize(b->root) != cudaSuccess)
    (void)cudaGetLastError();
  drop_batch_graph(b);
  for (auto& g : b->groups) {
    if (g->join) cudaEventDestroy(g->join);
    if (g->ready) cudaEventDestroy(g->ready);
    lp_destroy(g->ctx);
  }
  b->groups.clear();
  b->grouped = false;
}

// Merge the instances into groups (in order of first appearance) and tune them
// if the batch was asked to.
lp_status build_groups(lp_batch* b) {
  if (b->grouped) return LP_OK;
  drop_groups(b);
  for (size_t i = 0; i < b->inst.size(); ++i) {
    Inst& in = *b->inst[i];
    int g = -1;
    for (size_t j = 0; j < b->groups.size() && g < 0; ++j)
      if (same_group(b->inst[b->groups[j]->members[0]]->q, in.q)) g = static_cast<int>(j);
    if (g < 0) {
      b->groups.push_back(std::make_unique<Group>());
      g = static_cast<int>(b->groups.size()) - 1;
    }
    in.group = g;
    in.problem = static_cast<int>(b->groups[g]->members.size());
    b->groups[g]->members.push_back(static_cast<int>(i));
  }
  for (auto& gp : b->groups) {
    Group& g = *gp;
    std::vector<lp_ctx*> src;
    for (int i : g.members) {
      src.push_back(b->inst[i]->q.ctx);
      const std::vector<double>& y = b->inst[i]->q.y0;
      g.y0.insert(g.y0.end(), y.begin(), y.end());
    }
    lp_status st = lp_create(&g.ctx, b->device, 0, nullptr);
    if (st) {
      drop_groups(b);
      return bfail(b, st, lp_last_error(nullptr));
    }
    if (cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.ready, cudaEventDisableTiming) != cudaSuccess) {
      (void)cudaGetLastError();
      drop_groups(b);
      return bfail(b, LP_ERR_CUDA, "creating the group's events");
    }
    if ((st = lp::load_merged(g.ctx, src.data(), static_cast<int>(src.size()))) ||
        (b->tuned && (st = lp_autotune(g.ctx, b->inst[g.members[0]]->q.k, nullptr, nullptr, nullptr)))) {
      const std::string msg = lp_last_error(g.ctx);
      drop_groups(b);
      return bfail(b, st, msg);
    }
  }
  b->grouped = true;
  return LP_OK;
}

}  // namespace

extern "C" {

lp_status lp_batch_create(lp_batch** out, int device, size_t hbm_budget_bytes) {
  if (!out) return LP_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    (void)cudaGetLastError();
    return ndev == 0 ? LP_ERR_CUDA : LP_ERR_INVALID;
  }
  lp_batch* b = new (std::nothrow) lp_batch();
  if (!b) return LP_ERR_OOM;
  b->device = device;
  b->budget = hbm_budget_bytes;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    lp_batch_destroy(b);
    return LP_ERR_CUDA;
  }
  *out = b;
  return LP_OK;
}

lp_status lp_batch_add(lp_batch* b, const lp_request* q, int* index) {
  if (!b) return LP_ERR_INVALID;
  b->err.clear();
  if (!q || !index) return bfail(b, LP_ERR_INVALID, "request and index must be non-NULL");
  if (q->m < 1 || !q->rows || !q->parts || q->d < 1 || q->k < 1 || q->k > LP_MAX_K || q->k > q->d || !q->y0 ||
      q->T < 0 || q->refine_rounds < 0 || q->T + q->refine_rounds < 1 || (q->T > 0 && !q->p_schedule) ||
      (q->row_pitch != 0 && q->row_pitch < q->d) || (q->dtype == LP_FP8_E4M3 && !q->row_scales))
    return bfail(b, LP_ERR_INVALID, "malformed request");
  if (q->flags & LP_FLAG_TRACE) return bfail(b, LP_ERR_INVALID, "LP_FLAG_TRACE is not available in a batch");
  for (int t = 0; t < q->T; ++t)
    if (q->p_schedule[t] < 1) return bfail(b, LP_ERR_INVALID, "p_schedule entries must be >= 1");
  auto in = std::make_unique<Inst>();
  Request& r = in->q;
  r.m = q->m;
  r.d = q->d;
  r.pitch = q->row_pitch ? q->row_pitch : q->d;
  r.dtype = q->dtype;
  r.space = q->space;
  r.rows.assign(q->rows, q->rows + q->m);
  r.parts.assign(q->parts, q->parts + q->m);
  if (q->dtype == LP_FP8_E4M3) r.scales.assign(q->row_scales, q->row_scales + q->m);
  r.k = q->k;
  r.T = q->T;
  r.refine = q->refine_rounds;
  r.agg = q->agg;
  r.flags = q->flags;
  if (q->T > 0) r.sched.assign(q->p_schedule, q->p_schedule + q->T);
  r.y0.assign(q->y0, q->y0 + size_t(q->d) * q->k);
  r.est = lp::estimate_bytes(b->sms, r.m, r.rows.data(), r.d, r.pitch, r.dtype, r.k, r.space);
  // the instance's own copy and its share of its group's context
  if (b->budget && b->in_use + 2 * r.est > b->budget)
    return bfail(b, LP_ERR_OOM, "instance does not fit the batch's HBM budget");
  // the check a solve would make, now (a group would report it for all its instances)
  const int64_t smin = *std::min_element(r.rows.begin(), r.rows.end());
  if (smin < 1) return bfail(b, LP_ERR_INVALID, "a partition has no rows");
  if (r.k > smin) return bfail(b, LP_ERR_INVALID, "k exceeds the smallest partition");
  lp_status st = lp_create(&r.ctx, b->device, r.est, nullptr);
  if (st) return bfail(b, st, lp_last_error(nullptr));
  st = lp::load_pitched(r.ctx, r.m, r.rows.data(), r.d, r.pitch, r.dtype, r.parts.data(),
                        r.dtype == LP_FP8_E4M3 ? r.scales.data() : nullptr, r.space);
  if (st) {
    const std::string msg = lp_last_error(r.ctx);
    lp_destroy(r.ctx);
    return bfail(b, st, msg);
  }
  b->in_use += 2 * r.est;
  drop_groups(b);
  *index = static_cast<int>(b->inst.size());
  b->inst.push_back(std::move(in));
  return LP_OK;
}

lp_status lp_batch_autotune(lp_batch* b) {
  if (!b) return LP_ERR_INVALID;
  b->err.clear();
  if (b->inst.empty()) return bfail(b, LP_ERR_STATE, "empty batch");
  b->tuned = true;
  drop_groups(b);
  return build_groups(b);
}

lp_status lp_batch_solve(lp_batch* b) {
  if (!b) return LP_ERR_INVALID;
  b->err.clear();
  if (b->inst.empty()) return bfail(b, LP_ERR_STATE, "empty batch");
  if (cudaSetDevice(b->device) != cudaSuccess) {
    (void)cudaGetLastError();
    return bfail(b, LP_ERR_CUDA, "cudaSetDevice failed");
  }
  // the previous launch may still read the staged start blocks
  if (cudaStreamSynchronize(b->root) != cudaSuccess) {
    (void)cudaGetLastError();
    return bfail(b, LP_ERR_CUDA, "waiting for the previous batch solve");
  }
  b->solved = false;
  lp_status st = build_groups(b);
  if (st) return st;
  // start blocks in; the graph waits for every upload
  for (auto& gp : b->groups) {
    Group& g = *gp;
    const Request& r = b->inst[g.members[0]]->q;
    st = lp::batch_prepare(g.ctx, r.k, r.sched.empty() ? nullptr : r.sched.data(), r.T, r.agg, g.y0.data(), r.refine,
                           r.flags);
    if (st) return bfail(b, st, lp_last_error(g.ctx));
    if (cudaEventRecord(g.ready, lp::ctx_stream(g.ctx)) != cudaSuccess ||
        cudaStreamWaitEvent(b->root, g.ready, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      return bfail(b, LP_ERR_CUDA, "ordering the uploads");
    }
  }
  if (!b->exec) {
    cudaError_t e = cudaStreamBeginCapture(b->root, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->root);
    st = LP_OK;
    for (size_t i = 0; e == cudaSuccess && !st && i < b->groups.size(); ++i) {
      Group& g = *b->groups[i];
      const Request& r = b->inst[g.members[0]]->q;
      cudaStream_t s = lp::ctx_stream(g.ctx);
      e = cudaStreamWaitEvent(s, b->fork, 0);
      if (e != cudaSuccess) break;
      st = lp::batch_enqueue(g.ctx, r.k, r.sched.empty() ? nullptr : r.sched.data(), r.T, r.agg, r.refine, r.flags,
                             &g.captured);
      if (st) {
        b->err = lp_last_error(g.ctx);
        break;
      }
      e = cudaEventRecord(g.join, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->root, g.join, 0);
    }
    cudaGraph_t gr = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->root, &gr);
    if (st || e != cudaSuccess || ee != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      (void)cudaGetLastError();
      if (st) return st;
      return bfail(b, LP_ERR_CUDA, std::string("capturing the batch: ") +
                                       cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    e = cudaGraphInstantiate(&b->exec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      (void)cudaGetLastError();
      return bfail(b, LP_ERR_CUDA, std::string("instantiating the batch graph: ") + cudaGetErrorString(e));
    }
  }
  if (cudaGraphLaunch(b->exec, b->root) != cudaSuccess) {
    (void)cudaGetLastError();
    return bfail(b, LP_ERR_CUDA, "launching the batch graph");
  }
  for (auto& gp : b->groups) {
    const Request& r = b->inst[gp->members[0]]->q;
    lp::batch_mark(gp->ctx, r.k, gp->captured, r.T + r.refine, r.flags);
  }
  b->solved = true;
  return LP_OK;
}

lp_status lp_batch_result(lp_batch* b, int index, double* z_out, double* sigma_out, lp_stats* stats) {
  if (!b) return LP_ERR_INVALID;
  b->err.clear();
  if (index < 0 || index >= static_cast<int>(b->inst.size())) return bfail(b, LP_ERR_INVALID, "index out of range");
  if (!b->solved) return bfail(b, LP_ERR_STATE, "no batch solve to report");
  if (cudaStreamSynchronize(b->root) != cudaSuccess) {
    (void)cudaGetLastError();
    return bfail(b, LP_ERR_CUDA, "waiting for the batch");
  }
  const Inst& in = *b->inst[index];
  lp_ctx* c = b->groups[in.group]->ctx;
  const lp_status st = lp::problem_result(c, in.problem, z_out, sigma_out, stats);
  if (st) b->err = lp_last_error(c);
  return st;
}

int lp_batch_size(const lp_batch* b) { return b ? static_cast<int>(b->inst.size()) : 0; }

int lp_batch_groups(const lp_batch* b) { return b && b->grouped ? static_cast<int>(b->groups.size()) : 0; }

const char* lp_batch_error(const lp_batch* b) { return b ? b->err.c_str() : ""; }

void lp_batch_destroy(lp_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->root) cudaStreamSynchronize(b->root);
  drop_groups(b);
  for (auto& in : b->inst) lp_destroy(in->q.ctx);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->root) cudaStreamDestroy(b->root);
  delete b;
}

}  // extern "C"
