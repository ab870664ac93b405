// Serving form: continuous batching of nTT jobs on one GPU.
//
// Jobs arrive through ntt_server_submit (any thread) and wait in FIFO order.
// An engine thread admits the head of the queue while a job slot is free and
// the job's device footprint fits the HBM budget (an arena allocated once at
// creation), then advances every resident job in ticks: one tick is K
// multiplicative-update iterations of each resident job's current stage, all
// problems together in the grouped engine (one pass launch per shape bucket
// and one combine launch per iteration).  Stage boundaries fall on tick
// boundaries (K divides the stage's iteration count); at a boundary the job
// takes the column-L1 hand-off (W becomes core k, H scaled becomes the next
// unfolding) and draws the next stage's initial factors; after its last stage
// its cores are copied to the caller's host buffer and the job is done.
//
// Every problem's reductions run in an order fixed by its own shape (the
// engine's fixed split) and its initial factors come from its own seed, so a
// job's cores are bitwise the same whether it ran alone or among others.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "group_engine.cuh"
#include "serve_policy.h"

using namespace ntt;

namespace {

using Clock = std::chrono::steady_clock;

__global__ void cast_bf16_f32_kernel(const __nv_bfloat16* __restrict__ in, float* __restrict__ out, int64_t count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    out[i] = __bfloat162float(in[i]);
}

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

struct Job {
  int64_t id = 0;
  int d = 0;
  std::vector<int64_t> dims, ranks;
  std::vector<int64_t> m, n;          // per stage unfolding shape
  std::vector<int> r;
  const void* A = nullptr;            // caller's host tensor
  ntt_dtype dtype = NTT_F32;
  float* cores_host = nullptr;        // caller's host output
  uint64_t seed = 0;
  int state = NTT_JOB_QUEUED;
  ntt_status status = NTT_OK;
  int stage = 0, iters_done = 0;   // engine thread only
  int pub_stage = 0;               // stage as reported to callers (under the server lock)
  bool fresh = true;
  // device block and its layout (bytes from the block start)
  int64_t off = -1;
  size_t footprint = 0, o_x0 = 0, o_xbf = 0, o_h[2] = {0, 0}, o_cores = 0, o_scratch = 0, o_s = 0;
  std::vector<size_t> core_off;       // floats from the cores start
  size_t x_entries = 0, core_floats = 0;
  double t_submit = 0, t_admit = -1, t_done = -1;
};

}  // namespace

struct ntt_server_s {
  ntt_server_config cfg;
  int device = 0, sms = 0;
  char* arena_dev = nullptr;
  serve::Arena arena;
  serve::AdmissionQueue queue;
  std::unordered_map<int64_t, std::unique_ptr<Job>> jobs;
  std::vector<Job*> resident;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread engine;
  bool stop = false;
  cudaStream_t st = nullptr;
  char* tab_dev = nullptr;
  size_t tab_dev_bytes = 0;
  char* tab_host = nullptr;
  size_t tab_host_bytes = 0;
  int64_t next_id = 1;
  ntt_server_stats stats;
  Clock::time_point t0;
  double busy_s = 0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void run();
  ntt_status tick(std::vector<Job*>& fresh, std::vector<Job*>& done);
};

namespace {

// Stage s of job J: X, W (inside core s), H (ping-pong buffer, or the last core).
struct StagePtrs {
  const float* X;
  float* W;
  float* H;
};

StagePtrs stage_ptrs(ntt_server_s* S, const Job& J, int s) {
  char* base = S->arena_dev + J.off;
  float* cores = reinterpret_cast<float*>(base + J.o_cores);
  StagePtrs p;
  p.X = s == 0 ? reinterpret_cast<const float*>(base + J.o_x0)
               : reinterpret_cast<const float*>(base + J.o_h[(s - 1) & 1]);
  p.W = cores + J.core_off[s];
  p.H = s == J.d - 2 ? cores + J.core_off[J.d - 1] : reinterpret_cast<float*>(base + J.o_h[s & 1]);
  return p;
}

ntt_status init_stage(ntt_server_s* S, const Job& J, int s) {
  const StagePtrs p = stage_ptrs(S, J, s);
  if (launch_uniform(stream_key(J.seed, s, 0, 0), J.m[s] * J.r[s], p.W, S->st) != cudaSuccess ||
      launch_uniform(stream_key(J.seed, s, 0, 1), (int64_t)J.r[s] * J.n[s], p.H, S->st) != cudaSuccess)
    return NTT_ERR_CUDA;
  return NTT_OK;
}

// Shapes, feasibility and the device layout of a job; false when not servable.
ntt_status plan_job(Job& J, int sms) {
  if (J.d < 2 || J.d > NTT_MAX_D) return NTT_ERR_INVALID_ARG;
  if (J.ranks[0] != 1 || J.ranks[J.d] != 1) return NTT_ERR_INVALID_ARG;
  J.x_entries = 1;
  for (int k = 0; k < J.d; ++k) {
    if (J.dims[k] < 1) return NTT_ERR_INVALID_ARG;
    J.x_entries *= (size_t)J.dims[k];
  }
  size_t hmax[2] = {0, 0}, scratch = 0;
  J.core_off.assign(J.d, 0);
  J.core_floats = 0;
  for (int k = 0; k < J.d; ++k) {
    J.core_off[k] = J.core_floats;
    J.core_floats += (size_t)(J.ranks[k] * J.dims[k] * J.ranks[k + 1]);
  }
  for (int s = 0; s < J.d - 1; ++s) {
    int64_t n = 1;
    for (int k = s + 1; k < J.d; ++k) n *= J.dims[k];
    const int64_t m = J.ranks[s] * J.dims[s];
    const int64_t r = J.ranks[s + 1];
    if (r < 1 || r > m || r > n) return NTT_ERR_RANK_INFEASIBLE;
    if (r > NTT_MAX_RANK || m > NTT_MAX_TALL_ROWS) return NTT_ERR_UNSUPPORTED;
    J.m.push_back(m);
    J.n.push_back(n);
    J.r.push_back((int)r);
    if (s < J.d - 2) hmax[s & 1] = std::max(hmax[s & 1], (size_t)(r * n));
    GroupShape sh;
    sh.n = n;
    sh.m = (int)m;
    sh.re = (int)r;
    sh.blk = (int)r;
    scratch = std::max(scratch, group_problem_scratch(sh, sms));
  }
  size_t o = 0;
  J.o_x0 = o;
  o += a256(J.x_entries * 4);
  J.o_xbf = o;
  if (J.dtype == NTT_BF16) o += a256(J.x_entries * 2);
  J.o_h[0] = o;
  o += a256(hmax[0] * 4 + 4);
  J.o_h[1] = o;
  o += a256(hmax[1] * 4 + 4);
  J.o_cores = o;
  o += a256(J.core_floats * 4);
  J.o_s = o;
  o += a256(NTT_MAX_RANK * 4);
  J.o_scratch = o;
  o += a256(scratch);
  J.footprint = o;
  return NTT_OK;
}

}  // namespace

// One tick: copy in and initialise newly admitted jobs, K iterations of every
// resident job, hand-offs at stage ends, results of finished jobs to the host.
ntt_status ntt_server_s::tick(std::vector<Job*>& fresh, std::vector<Job*>& done) {
  for (Job* J : fresh) {
    char* base = arena_dev + J->off;
    float* x0 = reinterpret_cast<float*>(base + J->o_x0);
    if (J->dtype == NTT_BF16) {
      __nv_bfloat16* xb = reinterpret_cast<__nv_bfloat16*>(base + J->o_xbf);
      if (cudaMemcpyAsync(xb, J->A, J->x_entries * 2, cudaMemcpyHostToDevice, st) != cudaSuccess) return NTT_ERR_CUDA;
      const int grid = (int)std::min<int64_t>((int64_t)sms * 8, (J->x_entries + 1023) / 1024 + 1);
      cast_bf16_f32_kernel<<<grid, 256, 0, st>>>(xb, x0, (int64_t)J->x_entries);
      if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
    } else if (cudaMemcpyAsync(x0, J->A, J->x_entries * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      return NTT_ERR_CUDA;
    }
    ntt_status s = init_stage(this, *J, 0);
    if (s != NTT_OK) return s;
    J->fresh = false;
  }
  // K iterations of all resident problems
  std::vector<GroupShape> shapes;
  std::vector<GroupPtrs> ptrs;
  for (Job* J : resident) {
    const int s = J->stage;
    GroupShape sh;
    sh.n = J->n[s];
    sh.m = (int)J->m[s];
    sh.re = J->r[s];
    sh.blk = J->r[s];
    shapes.push_back(sh);
    const StagePtrs p = stage_ptrs(this, *J, s);
    GroupPtrs g;
    g.X = p.X;
    g.W = p.W;
    g.H = p.H;
    g.scratch = arena_dev + J->off + J->o_scratch;
    ptrs.push_back(g);
  }
  GroupPlan pl;
  ntt_status s = group_plan(shapes, sms, 0, true, false, &pl);
  if (s != NTT_OK) return s;
  if (pl.bytes > tab_dev_bytes) {
    if (tab_dev) cudaFree(tab_dev);
    tab_dev = nullptr;
    tab_dev_bytes = 0;
    if (cudaMalloc(&tab_dev, pl.bytes * 2) != cudaSuccess) return NTT_ERR_OOM;
    tab_dev_bytes = pl.bytes * 2;
  }
  if (pl.table_bytes > tab_host_bytes) {
    if (tab_host) cudaFreeHost(tab_host);
    tab_host = nullptr;
    tab_host_bytes = 0;
    if (cudaMallocHost(&tab_host, pl.table_bytes * 2) != cudaSuccess) return NTT_ERR_OOM;
    tab_host_bytes = pl.table_bytes * 2;
  }
  s = group_run(pl, ptrs.data(), tab_dev, tab_host, cfg.tick_iters, cfg.eps_mu, st);
  if (s != NTT_OK) return s;
  // stage ends
  for (Job* J : resident) {
    J->iters_done += cfg.tick_iters;
    if (J->iters_done < cfg.stage_iters) continue;
    const int st_k = J->stage;
    const StagePtrs p = stage_ptrs(this, *J, st_k);
    float* sbuf = reinterpret_cast<float*>(arena_dev + J->off + J->o_s);
    if (launch_handoff(p.W, p.H, J->m[st_k], J->n[st_k], J->r[st_k], sbuf, st) != cudaSuccess) return NTT_ERR_CUDA;
    J->stage += 1;
    J->iters_done = 0;
    if (J->stage == J->d - 1) {
      const float* cores = reinterpret_cast<const float*>(arena_dev + J->off + J->o_cores);
      if (cudaMemcpyAsync(J->cores_host, cores, J->core_floats * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return NTT_ERR_CUDA;
      done.push_back(J);
    } else {
      s = init_stage(this, *J, J->stage);
      if (s != NTT_OK) return s;
    }
  }
  return cudaStreamSynchronize(st) == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

void ntt_server_s::run() {
  cudaSetDevice(device);
  while (true) {
    std::vector<Job*> fresh, done;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] {
        return stop || !resident.empty() || (!queue.empty() && (int)resident.size() < cfg.max_jobs);
      });
      if (stop) return;
      const double t = now();
      queue.admit(
          arena, cfg.max_jobs - (int)resident.size(),
          [&](int64_t id, int64_t off) {
            Job* J = jobs[id].get();
            J->off = off;
            J->state = NTT_JOB_RUNNING;
            J->t_admit = t;
            resident.push_back(J);
            fresh.push_back(J);
          },
          [&](int64_t id) {
            Job* J = jobs[id].get();
            J->state = NTT_JOB_FAILED;
            J->status = NTT_ERR_OOM;
            J->t_done = t;
            stats.failed += 1;
            cv_done.notify_all();
          });
      if (resident.empty()) continue;
    }
    const double t_start = now();
    const ntt_status s = tick(fresh, done);
    const double t_end = now();
    std::lock_guard<std::mutex> lk(mu);
    busy_s += t_end - t_start;
    stats.ticks += 1;
    if (s != NTT_OK) {
      // the device work of this tick is unusable: fail every resident job
      cudaStreamSynchronize(st);
      cudaGetLastError();
      for (Job* J : resident) {
        J->state = NTT_JOB_FAILED;
        J->status = s;
        J->t_done = t_end;
        arena.release(J->off);
        stats.failed += 1;
      }
      resident.clear();
    } else {
      for (Job* J : resident) J->pub_stage = J->stage;
      for (Job* J : done) {
        J->state = NTT_JOB_DONE;
        J->t_done = t_end;
        arena.release(J->off);
        stats.completed += 1;
        for (size_t i = 0; i < resident.size(); ++i)
          if (resident[i] == J) {
            resident.erase(resident.begin() + i);
            break;
          }
      }
    }
    cv_done.notify_all();
  }
}

namespace {

void fill_info(const Job& J, ntt_job_info* info) {
  if (!info) return;
  info->state = J.state;
  info->status = J.status;
  info->stage = J.pub_stage;
  info->t_submit = J.t_submit;
  info->t_admit = J.t_admit;
  info->t_done = J.t_done;
  info->footprint_bytes = J.footprint;
}

}  // namespace

extern "C" {

ntt_status ntt_server_create(const ntt_server_config* cfg, ntt_server* out) {
  if (!cfg || !out) return NTT_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->hbm_budget_bytes < (1u << 20) || cfg->max_jobs < 1 || cfg->tick_iters < 1 || cfg->stage_iters < 1 ||
      cfg->stage_iters % cfg->tick_iters != 0 || !(cfg->eps_mu >= 0.0f))
    return NTT_ERR_INVALID_ARG;
  ntt_server S = new (std::nothrow) ntt_server_s();
  if (!S) return NTT_ERR_OOM;
  S->cfg = *cfg;
  std::memset(&S->stats, 0, sizeof(S->stats));
  S->t0 = Clock::now();
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return NTT_ERR_CUDA;
  }
  S->sms = device_sms();
  if (cudaMalloc(&S->arena_dev, cfg->hbm_budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return NTT_ERR_OOM;
  }
  S->arena.reset(cfg->hbm_budget_bytes);
  if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(S->arena_dev);
    cudaGetLastError();
    delete S;
    return NTT_ERR_CUDA;
  }
  S->engine = std::thread([S] { S->run(); });
  *out = S;
  return NTT_OK;
}

ntt_status ntt_server_job_footprint(int d, const int64_t* dims, const int64_t* ranks, ntt_dtype dtype,
                                    size_t* bytes) {
  if (!dims || !ranks || !bytes || d < 2 || d > NTT_MAX_D || (dtype != NTT_F32 && dtype != NTT_BF16))
    return NTT_ERR_INVALID_ARG;
  Job J;
  J.d = d;
  J.dims.assign(dims, dims + d);
  J.ranks.assign(ranks, ranks + d + 1);
  J.dtype = dtype;
  const ntt_status s = plan_job(J, device_sms());
  if (s != NTT_OK) return s;
  *bytes = J.footprint;
  return NTT_OK;
}

ntt_status ntt_server_submit(ntt_server S, int d, const int64_t* dims, const int64_t* ranks, const void* A_host,
                             ntt_dtype dtype, uint64_t seed, float* cores_host, int64_t* job_id) {
  if (!S || !dims || !ranks || !A_host || !cores_host || !job_id || d < 2 || d > NTT_MAX_D ||
      (dtype != NTT_F32 && dtype != NTT_BF16))
    return NTT_ERR_INVALID_ARG;
  std::unique_ptr<Job> J(new (std::nothrow) Job());
  if (!J) return NTT_ERR_OOM;
  J->d = d;
  J->dims.assign(dims, dims + d);
  J->ranks.assign(ranks, ranks + d + 1);
  J->A = A_host;
  J->dtype = dtype;
  J->cores_host = cores_host;
  J->seed = seed;
  const ntt_status s = plan_job(*J, S->sms);
  if (s != NTT_OK) return s;
  std::lock_guard<std::mutex> lk(S->mu);
  if (J->footprint > S->arena.capacity()) return NTT_ERR_OOM;
  J->id = S->next_id++;
  J->t_submit = S->now();
  *job_id = J->id;
  S->queue.push(J->id, J->footprint);
  S->jobs[J->id] = std::move(J);
  S->stats.submitted += 1;
  S->cv_work.notify_one();
  return NTT_OK;
}

ntt_status ntt_server_poll(ntt_server S, int64_t job_id, ntt_job_info* info) {
  if (!S || !info) return NTT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return NTT_ERR_INVALID_ARG;
  fill_info(*it->second, info);
  return NTT_OK;
}

ntt_status ntt_server_wait(ntt_server S, int64_t job_id, double timeout_s, ntt_job_info* info) {
  if (!S) return NTT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return NTT_ERR_INVALID_ARG;
  Job* J = it->second.get();
  auto finished = [&] { return J->state == NTT_JOB_DONE || J->state == NTT_JOB_FAILED; };
  if (timeout_s < 0) {
    S->cv_done.wait(lk, finished);
  } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), finished)) {
    fill_info(*J, info);
    return NTT_ERR_TIMEOUT;
  }
  fill_info(*J, info);
  const ntt_status st = J->status;
  S->jobs.erase(it);   // the result is the caller's now
  return st;
}

ntt_status ntt_server_get_stats(ntt_server S, ntt_server_stats* out) {
  if (!S || !out) return NTT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  out->resident = (int)S->resident.size();
  out->queued = (int)S->queue.size();
  out->bytes_in_use = S->arena.in_use();
  out->peak_bytes = S->arena.peak();
  out->capacity_bytes = S->arena.capacity();
  out->busy_s = S->busy_s;
  return NTT_OK;
}

ntt_status ntt_server_destroy(ntt_server S) {
  if (!S) return NTT_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->engine.joinable()) S->engine.join();
  if (S->st) {
    cudaStreamSynchronize(S->st);
    cudaStreamDestroy(S->st);
  }
  if (S->arena_dev) cudaFree(S->arena_dev);
  if (S->tab_dev) cudaFree(S->tab_dev);
  if (S->tab_host) cudaFreeHost(S->tab_host);
  cudaGetLastError();
  delete S;
  return NTT_OK;
}

}  // extern "C"
