// Serving loop: continuous batching of independent Carreau-Stokes solves on one GPU under a
// device-memory budget.  Each slot is a worker thread with its own CUDA stream; a request is
// analysed on the host (symbolic set-up: exact sizes and a memory estimate), admitted when
// the estimate fits in the budget, set up and solved on the slot's stream, and released.
// Requests arriving while others run are admitted as memory frees up, and the kernels of the
// requests in flight overlap on the device.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "common.h"
#include "kernels.h"
#include "setup.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// a request with private copies of every host input
struct Job {
  gdsw_request req{};
  std::vector<uint8_t> mask, tags;
  std::vector<double> g, uk, rhs;
  std::vector<int32_t> part, grp0, grp1;
  gdsw_request_status st{};
  double t_submit = 0, t_admit = 0;
  std::string err;
};

}  // namespace

struct gdsw_server {
  int device = 0;
  int64_t budget = 0;
  int slots = 1;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, std::unique_ptr<Job>> jobs;
  int64_t next = 1;
  int64_t used = 0;
  bool stop = false;
  gdsw_server_stats stats{};
};

namespace {

void run_job(gdsw_server* S, int slot, Job& J) {
  using namespace gdsw;
  gdsw_ctx* c = new gdsw_ctx();
  double* d_b = nullptr;
  double* d_x = nullptr;
  int64_t reserved = 0;
  try {
    // host symbolic analysis: sizes and the admission estimate
    c->host_only = true;
    setup_impl(c, &J.req.mesh, &J.req.visc, &J.req.part, &J.req.levels, &J.req.opt);
    const int64_t n = c->mesh.n;
    GDSW_CHECK(J.req.x_len == n, GDSW_ERR_INVALID_ARG, "x_len differs from the problem size");
    const int64_t est = c->est_device_bytes + 16 * n + (int64_t(64) << 20);
    {
      std::unique_lock<std::mutex> lk(S->mu);
      J.st.n = n;
      J.st.est_bytes = est;
      GDSW_CHECK(est <= S->budget, GDSW_ERR_OOM, "request does not fit in the server's memory budget");
      J.st.state = GDSW_REQ_WAITING;
      S->cv.wait(lk, [&] { return S->used + est <= S->budget; });
      S->used += est;
      reserved = est;
      S->stats.peak_used_bytes = std::max(S->stats.peak_used_bytes, S->used);
      S->stats.running++;
      S->stats.peak_running = std::max(S->stats.peak_running, S->stats.running);
      J.st.state = GDSW_REQ_RUNNING;
      J.st.slot = slot;
      J.t_admit = now_ms();
      J.st.queue_ms = J.t_admit - J.t_submit;
    }
    // device set-up on the slot's stream
    gdsw_options o = J.req.opt;
    o.stream = S->streams[slot];
    c->host_only = false;
    double t0 = now_ms();
    setup_impl(c, &J.req.mesh, &J.req.visc, &J.req.part, &J.req.levels, &o);
    double t1 = now_ms();
    cudaStream_t s = S->streams[slot];
    GDSW_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d_b), 8 * n, s));  // stream-ordered: no device-wide sync
    GDSW_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d_x), 8 * n, s));
    if (!J.rhs.empty())
      GDSW_CUDA(cudaMemcpyAsync(d_b, J.rhs.data(), 8 * n, cudaMemcpyHostToDevice, s));
    else
      launch_lift(c, d_b, s);
    GDSW_CUDA(cudaMemsetAsync(d_x, 0, 8 * n, s));
    gdsw_solve_info info{};
    fgmres_solve(c, d_b, d_x, &info);
    GDSW_CUDA(cudaMemcpyAsync(J.req.x, d_x, 8 * n, cudaMemcpyDeviceToHost, s));
    GDSW_CUDA(cudaStreamSynchronize(s));
    double t2 = now_ms();
    cudaFreeAsync(d_b, s);
    cudaFreeAsync(d_x, s);
    d_b = d_x = nullptr;
    gdsw_destroy(c);
    c = nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= reserved;
    S->stats.running--;
    J.st.iterations = info.iterations;
    J.st.relres = info.relres;
    J.st.status = info.status;
    J.st.setup_ms = t1 - t0;
    J.st.solve_ms = t2 - t1;
    J.st.latency_ms = t2 - J.t_submit;
    J.st.state = (info.status == GDSW_OK || info.status == GDSW_ERR_NOT_CONVERGED) ? GDSW_REQ_DONE : GDSW_REQ_FAILED;
    if (J.st.state == GDSW_REQ_DONE) S->stats.completed++;
    else S->stats.failed++;
  } catch (const gdsw::Error& e) {
    if (d_b) cudaFreeAsync(d_b, S->streams[slot]);
    if (d_x) cudaFreeAsync(d_x, S->streams[slot]);
    if (d_b || d_x) cudaStreamSynchronize(S->streams[slot]);
    if (c) gdsw_destroy(c);
    std::lock_guard<std::mutex> lk(S->mu);
    if (reserved) {
      S->used -= reserved;
      S->stats.running--;
    }
    J.err = e.msg;
    J.st.status = e.code;
    J.st.state = GDSW_REQ_FAILED;
    J.st.latency_ms = now_ms() - J.t_submit;
    S->stats.failed++;
  }
  S->cv.notify_all();
}

void worker(gdsw_server* S, int slot) {
  cudaSetDevice(S->device);
  while (true) {
    Job* J = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      if (S->queue.empty()) return;  // stop requested and nothing left to do
      int64_t t = S->queue.front();
      S->queue.pop_front();
      J = S->jobs[t].get();
      J->st.state = GDSW_REQ_ANALYSING;
    }
    run_job(S, slot, *J);
  }
}

template <typename T>
std::vector<T> copy_of(const T* p, int64_t n) {
  return p ? std::vector<T>(p, p + n) : std::vector<T>();
}

}  // namespace

extern "C" {

int gdsw_server_create(int32_t device, int64_t mem_budget_bytes, int32_t max_slots, gdsw_server** out) {
  if (!out || mem_budget_bytes <= 0 || max_slots < 1 || max_slots > 64) return GDSW_ERR_INVALID_ARG;
  *out = nullptr;
  gdsw_server* S = new (std::nothrow) gdsw_server();
  if (!S) return GDSW_ERR_OOM;
  S->device = device;
  S->budget = mem_budget_bytes;
  S->slots = max_slots;
  S->stats.budget_bytes = mem_budget_bytes;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete S;
    return GDSW_ERR_CUDA;
  }
  for (int q = 0; q < max_slots; ++q) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t t : S->streams) cudaStreamDestroy(t);
      delete S;
      return GDSW_ERR_CUDA;
    }
    S->streams.push_back(s);
  }
  for (int q = 0; q < max_slots; ++q) S->workers.emplace_back(worker, S, q);
  *out = S;
  return GDSW_OK;
}

int gdsw_server_submit(gdsw_server* S, const gdsw_request* r, int64_t* ticket) {
  if (!S || !r || !ticket || !r->x || r->x_len <= 0 || !r->mesh.mask || !r->mesh.tags || !r->mesh.g ||
      !r->part.elem_part || r->part.n_groups < 0 || r->part.n_groups > 2)
    return GDSW_ERR_INVALID_ARG;
  auto J = std::make_unique<Job>();
  const gdsw_mesh& m = r->mesh;
  const int64_t ne = int64_t(m.nx) * m.ny * m.nz;
  const int64_t nn = int64_t(2 * m.nx + 1) * (2 * m.ny + 1) * (2 * m.nz + 1);
  try {
    J->req = *r;
    J->mask = copy_of(m.mask, ne);
    J->tags = copy_of(m.tags, nn);
    J->g = copy_of(m.g, 3 * nn);
    J->uk = copy_of(r->visc.uk, 3 * nn);
    J->part = copy_of(r->part.elem_part, ne);
    if (r->part.n_groups > 0) J->grp0 = copy_of(r->part.groups[0], r->part.group_len[0]);
    if (r->part.n_groups > 1) J->grp1 = copy_of(r->part.groups[1], r->part.group_len[1]);
    J->rhs = copy_of(r->rhs, r->x_len);
  } catch (const std::bad_alloc&) {
    return GDSW_ERR_OOM;
  }
  J->req.mesh.mask = J->mask.data();
  J->req.mesh.tags = J->tags.data();
  J->req.mesh.g = J->g.data();
  J->req.visc.uk = r->visc.uk ? J->uk.data() : nullptr;
  J->req.part.elem_part = J->part.data();
  J->req.part.groups[0] = J->grp0.empty() ? nullptr : J->grp0.data();
  J->req.part.groups[1] = J->grp1.empty() ? nullptr : J->grp1.data();
  J->req.rhs = nullptr;
  J->st.state = GDSW_REQ_QUEUED;
  J->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return GDSW_ERR_INVALID_ARG;
    *ticket = S->next++;
    S->jobs[*ticket] = std::move(J);
    S->queue.push_back(*ticket);
    S->stats.submitted++;
  }
  S->cv.notify_all();
  return GDSW_OK;
}

int gdsw_server_poll(gdsw_server* S, int64_t ticket, gdsw_request_status* st) {
  if (!S || !st) return GDSW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return GDSW_ERR_INVALID_ARG;
  *st = it->second->st;
  return GDSW_OK;
}

int gdsw_server_wait(gdsw_server* S, int64_t ticket, gdsw_request_status* st) {
  if (!S || !st) return GDSW_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return GDSW_ERR_INVALID_ARG;
  Job* J = it->second.get();
  S->cv.wait(lk, [&] { return J->st.state == GDSW_REQ_DONE || J->st.state == GDSW_REQ_FAILED; });
  *st = J->st;
  return GDSW_OK;
}

int gdsw_server_stats_read(gdsw_server* S, gdsw_server_stats* st) {
  if (!S || !st) return GDSW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *st = S->stats;
  st->used_bytes = S->used;
  return GDSW_OK;
}

int gdsw_server_destroy(gdsw_server* S) {
  if (!S) return GDSW_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& w : S->workers) w.join();
  for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
  delete S;
  return GDSW_OK;
}

}  // extern "C"
