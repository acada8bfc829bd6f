// serve.cu -- served dynamic rebuilds: the time step of a resident point
// system (counter-based Gaussian displacement with wall reflection), result
// digests, and the continuous-batching server of include/fmmds.h.
//
// Dynamic problems rebuild the FMM structures at every time step (Sec. 1).
// The server keeps each system's points on the device; a worker thread per
// context takes every system that is waiting when it frees up, moves its
// points one step and rebuilds all of them in one batched build
// (fmm_build_batched), so the launch cost of many small rebuilds is shared
// and the builds of different workers overlap on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {
namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4.1): ten rounds of
// two 32 x 32 -> 64-bit multiplies that mix the four counter words, with the
// key bumped by the Weyl increments between rounds.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = kPhiloxM0 * c.x, hi0 = __umulhi(kPhiloxM0, c.x);
    const uint32_t lo1 = kPhiloxM1 * c.z, hi1 = __umulhi(kPhiloxM1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

// (floor(r / 2^9) + 1/2) * 2^-23: exact in float32, strictly inside (0, 1).
__device__ __forceinline__ float unit_open(uint32_t r) {
  return ((float)(r >> 9) + 0.5f) * 0x1p-23f;
}

__device__ __forceinline__ float reflect_unit(float x) {
  x = x < 0.f ? -x : x;
  return x > 1.f ? 2.f - x : x;
}

__global__ void __launch_bounds__(256) displace_kernel(float* __restrict__ xyz, uint32_t n,
                                                       uint32_t k0, uint32_t k1, uint32_t step_lo,
                                                       uint32_t step_hi, float sigma) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint4 r = philox4x32_10(make_uint4(i, step_lo, step_hi, 0u), k0, k1);
    const float rad0 = sqrtf(-2.f * logf(unit_open(r.x)));
    const float rad1 = sqrtf(-2.f * logf(unit_open(r.z)));
    float s1, c1;
    sincospif(2.f * unit_open(r.y), &s1, &c1);
    const float c3 = cospif(2.f * unit_open(r.w));
    float* p = xyz + 3ull * i;
    p[0] = reflect_unit(fmaf(sigma, rad0 * c1, p[0]));
    p[1] = reflect_unit(fmaf(sigma, rad0 * s1, p[1]));
    p[2] = reflect_unit(fmaf(sigma, rad1 * c3, p[2]));
  }
}

int launch_displace(float* xyz, uint32_t n, uint64_t seed, uint64_t step, float sigma,
                    cudaStream_t s) {
  if (n == 0) return FMM_OK;
  uint32_t grid = (n + 255) / 256;
  if (grid > 152u * 16u) grid = 152u * 16u;
  displace_kernel<<<grid, 256, 0, s>>>(xyz, n, (uint32_t)seed, (uint32_t)(seed >> 32),
                                       (uint32_t)step, (uint32_t)(step >> 32), sigma);
  return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

// Domain check of points added to the server (every coordinate in [0, 1]).
__global__ void check_unit_kernel(const float* __restrict__ xyz, uint64_t count, uint32_t* bad) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const float v = xyz[i];
    if (!(v >= 0.f && v <= 1.f)) atomicExch(bad, 1u);
  }
}

// ---------------------------------------------------------------------------
// Digest of an array: sum over elements of a 64-bit mix of (tag, index,
// value), so equal arrays give equal digests whatever the thread order.  The
// mix is the finaliser of SplitMix64 (Steele, Lea, Flood, OOPSLA'14).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256) digest_kernel(const void* __restrict__ p, uint64_t count,
                                                     uint32_t elem, uint64_t tag,
                                                     unsigned long long* acc) {
  uint64_t h = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t v = elem == 8 ? static_cast<const uint64_t*>(p)[i]
                                 : (uint64_t) static_cast<const uint32_t*>(p)[i];
    h += mix64(mix64(tag * 0x9E3779B97F4A7C15ull + i) ^ v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31) == 0 && h) atomicAdd(acc, (unsigned long long)h);
}

void digest_array(const void* p, uint64_t count, uint32_t elem, uint64_t tag,
                  unsigned long long* acc, cudaStream_t s) {
  if (!p || count == 0) return;
  uint64_t grid = (count + 255) / 256;
  if (grid > 152u * 8u) grid = 152u * 8u;
  digest_kernel<<<(uint32_t)grid, 256, 0, s>>>(p, count, elem, tag, acc);
}

// Every output array of one tree, each under its own tag.
void digest_tree(const fmm_tree& t, unsigned long long* acc, cudaStream_t s) {
  uint64_t tag = 1;
  digest_array(t.perm_src, t.n_src, 4, tag++, acc, s);
  digest_array(t.perm_recv, t.n_recv, 4, tag++, acc, s);
  for (int l = 0; l <= t.L; ++l) {
    const uint32_t nb[2] = {t.nbox_src[l], t.nbox_recv[l]};
    const uint64_t* key[2] = {t.key_src[l], t.key_recv[l]};
    const uint32_t* off[2] = {t.off_src[l], t.off_recv[l]};
    const uint32_t* par[2] = {t.parent_src[l], t.parent_recv[l]};
    const uint32_t* chi[2] = {t.child_src[l], t.child_recv[l]};
    for (int k = 0; k < 2; ++k) {
      digest_array(key[k], nb[k], 8, 100 * l + 10 * k + 1, acc, s);
      digest_array(off[k], (uint64_t)nb[k] + 1, 4, 100 * l + 10 * k + 2, acc, s);
      if (l >= 1) digest_array(par[k], nb[k], 4, 100 * l + 10 * k + 3, acc, s);
      if (l < t.L) digest_array(chi[k], (uint64_t)nb[k] + 1, 4, 100 * l + 10 * k + 4, acc, s);
    }
    if (l >= 2) {
      digest_array(t.e2_off[l], (uint64_t)t.nbox_recv[l] + 1, 4, 100 * l + 5, acc, s);
      digest_array(t.e2_idx[l], t.nnz_e2[l], 4, 100 * l + 6, acc, s);
      digest_array(t.e4_off[l], (uint64_t)t.nbox_recv[l] + 1, 4, 100 * l + 7, acc, s);
      digest_array(t.e4_idx[l], t.nnz_e4[l], 4, 100 * l + 8, acc, s);
    }
  }
}

// ---------------------------------------------------------------------------
// Server.

using Clock = std::chrono::steady_clock;

struct Request {
  fmm_request_info info{};
  bool done = false;
};

struct System {
  float* xyz = nullptr;  // device, owned
  uint32_t n = 0;
  int L = 0;
  float sigma = 0.f;
  uint64_t seed = 0;
  uint64_t step = 0;
  uint64_t est = 0;  // workspace estimate of one build
  bool busy = false;
  std::deque<uint64_t> queue;  // waiting request ids, arrival order
  fmm_tree last{};
  bool has_last = false;
  uint32_t last_worker = 0;  // the worker whose arena holds `last` ...
  uint64_t last_gen = 0;     // ... while its batch count is still this
};

struct Worker {
  fmm_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  unsigned long long* digest = nullptr;  // device accumulators, one per batch slot
  uint64_t gen = 0;                      // batches taken (each one reuses the arena)
  std::thread th;
};

}  // namespace
}  // namespace fmm

struct fmm_server {
  int device = 0;
  fmm_server_params prm{};
  uint64_t budget = 0;  // per worker
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  bool stop = false;
  std::deque<fmm::System> systems;  // stable references: workers hold one outside the lock
  std::vector<std::unique_ptr<fmm::Request>> reqs;  // by id
  std::vector<fmm::Worker> workers;
  // fmm_server_tree's rebuilds of systems whose worker has built again
  fmm_ctx* qctx = nullptr;
  cudaStream_t qstream = nullptr;
};

namespace fmm {
namespace {

double now_s(const fmm_server* S) {
  return std::chrono::duration<double>(Clock::now() - S->t0).count();
}

bool any_ready(const fmm_server* S) {
  for (auto& y : S->systems)
    if (!y.busy && !y.queue.empty()) return true;
  return false;
}

// Under the lock: the worker's next batch -- waiting systems, oldest request
// first, at most max_batch, while their estimates fit the budget.
void take_batch(fmm_server* S, std::vector<uint32_t>* sys, std::vector<uint64_t>* ids) {
  sys->clear();
  ids->clear();
  std::vector<uint32_t> ready;
  for (uint32_t i = 0; i < S->systems.size(); ++i)
    if (!S->systems[i].busy && !S->systems[i].queue.empty()) ready.push_back(i);
  std::sort(ready.begin(), ready.end(), [&](uint32_t a, uint32_t b) {
    const double ta = S->reqs[S->systems[a].queue.front()]->info.t_arrival;
    const double tb = S->reqs[S->systems[b].queue.front()]->info.t_arrival;
    return ta != tb ? ta < tb : a < b;
  });
  uint64_t used = 0;
  const double t = now_s(S);
  for (uint32_t i : ready) {
    if (sys->size() >= S->prm.max_batch) break;
    System& y = S->systems[i];
    if (!sys->empty() && used + y.est > S->budget) continue;
    used += y.est;
    y.busy = true;
    const uint64_t id = y.queue.front();
    y.queue.pop_front();
    S->reqs[id]->info.t_start = t;
    sys->push_back(i);
    ids->push_back(id);
  }
}

void worker_main(fmm_server* S, uint32_t w) {
  cudaSetDevice(S->device);
  Worker& W = S->workers[w];
  std::vector<uint32_t> sys;
  std::vector<uint64_t> ids;
  std::vector<fmm_set> sets;
  std::vector<fmm_tree> outs;
  std::vector<unsigned long long> dig;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->work_cv.wait(lk, [&] { return S->stop || any_ready(S); });
      if (!any_ready(S)) return;  // stopping, nothing left that this worker can take
      take_batch(S, &sys, &ids);
      ++W.gen;  // the trees of this worker's previous batch are about to be overwritten
    }
    const uint32_t k = (uint32_t)sys.size();
    int st = FMM_OK;
    sets.assign(k, fmm_set{});
    outs.assign(k, fmm_tree{});
    // Systems whose time step was launched: only they move on a step, so
    // that a system's points stay a function of (seed, step) even when a
    // launch fails partway through the batch.
    uint32_t moved = 0;
    for (uint32_t j = 0; j < k && st == FMM_OK; ++j) {
      System& y = S->systems[sys[j]];  // busy: only this worker touches it
      st = launch_displace(y.xyz, y.n, y.seed, y.step, y.sigma, W.stream);
      if (st == FMM_OK) moved = j + 1;
      sets[j] = fmm_set{y.xyz, y.n, y.xyz, y.n, y.L};
    }
    if (st == FMM_OK) {
      fmm_params p{0, 0, 0, 0};
      st = fmm_build_batched(W.ctx, sets.data(), k, p, outs.data(), W.stream);
    }
    dig.assign(k, 0ull);
    if (st == FMM_OK && (S->prm.flags & FMM_SERVER_DIGEST)) {
      if (cudaMemsetAsync(W.digest, 0, sizeof(unsigned long long) * k, W.stream) != cudaSuccess)
        st = FMM_ERR_CUDA;
      for (uint32_t j = 0; j < k && st == FMM_OK; ++j) digest_tree(outs[j], W.digest + j, W.stream);
      if (st == FMM_OK &&
          (cudaMemcpyAsync(dig.data(), W.digest, sizeof(unsigned long long) * k,
                           cudaMemcpyDeviceToHost, W.stream) != cudaSuccess ||
           cudaStreamSynchronize(W.stream) != cudaSuccess))
        st = FMM_ERR_CUDA;
    }
    if (st != FMM_OK) {
      cudaStreamSynchronize(W.stream);
      cudaGetLastError();
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const double t = now_s(S);
      for (uint32_t j = 0; j < k; ++j) {
        System& y = S->systems[sys[j]];
        fmm_request_info& inf = S->reqs[ids[j]]->info;
        if (j < moved) y.step += 1;
        y.busy = false;
        y.last = outs[j];
        y.has_last = st == FMM_OK;
        y.last_worker = w;
        y.last_gen = W.gen;
        inf.status = (uint32_t)st;
        inf.step = y.step;
        inf.t_done = t;
        inf.batch_size = k;
        inf.worker = w;
        inf.points = y.n;
        inf.nnz_e2 = inf.nnz_e4 = 0;
        if (st == FMM_OK)
          for (int l = 2; l <= outs[j].L; ++l) {
            inf.nnz_e2 += outs[j].nnz_e2[l];
            inf.nnz_e4 += outs[j].nnz_e4[l];
          }
        inf.digest = dig[j];
        S->reqs[ids[j]]->done = true;
      }
    }
    S->work_cv.notify_all();
    S->done_cv.notify_all();
  }
}

// Under the lock: a new request of `system` arriving at time t.
uint64_t enqueue(fmm_server* S, uint32_t system, double t) {
  const uint64_t id = S->reqs.size();
  auto r = std::make_unique<Request>();
  r->info.id = id;
  r->info.system = system;
  r->info.t_arrival = t;
  S->reqs.push_back(std::move(r));
  S->systems[system].queue.push_back(id);
  return id;
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" {

int fmm_displace(float* xyz, uint32_t n, uint64_t seed, uint64_t step, float sigma, void* stream) {
  if (n > 0 && !xyz) return FMM_ERR_ARG;
  return launch_displace(xyz, n, seed, step, sigma, static_cast<cudaStream_t>(stream));
}

int fmm_server_create(fmm_server** srv, int device, const fmm_server_params* params) {
  if (!srv || !params || params->workers == 0 || params->max_batch == 0 ||
      (params->flags & ~FMM_SERVER_DIGEST))
    return FMM_ERR_ARG;
  *srv = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return FMM_ERR_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  auto S = std::make_unique<fmm_server>();
  S->device = device;
  S->prm = *params;
  S->t0 = Clock::now();
  uint64_t budget = params->mem_budget;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      cudaSetDevice(prev);
      return FMM_ERR_CUDA;
    }
    budget = (uint64_t)(0.8 * (double)fr);
  }
  S->budget = budget / params->workers;
  S->workers.resize(params->workers);
  int st = FMM_OK;
  for (auto& W : S->workers) {
    if (fmm_create(&W.ctx, device, nullptr, nullptr, nullptr) != FMM_OK ||
        cudaStreamCreateWithFlags(&W.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&W.digest, sizeof(unsigned long long) * params->max_batch) != cudaSuccess) {
      cudaGetLastError();
      st = FMM_ERR_CUDA;
      break;
    }
  }
  if (st != FMM_OK) {
    for (auto& W : S->workers) {
      if (W.ctx) fmm_destroy(W.ctx);
      if (W.stream) cudaStreamDestroy(W.stream);
      if (W.digest) cudaFree(W.digest);
    }
    cudaSetDevice(prev);
    return st;
  }
  fmm_server* raw = S.release();
  for (uint32_t w = 0; w < raw->workers.size(); ++w)
    raw->workers[w].th = std::thread(worker_main, raw, w);
  cudaSetDevice(prev);
  *srv = raw;
  return FMM_OK;
}

int fmm_server_destroy(fmm_server* S) {
  if (!S) return FMM_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->work_cv.notify_all();
  for (auto& W : S->workers)
    if (W.th.joinable()) W.th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  if (S->qctx) fmm_destroy(S->qctx);
  if (S->qstream) cudaStreamDestroy(S->qstream);
  for (auto& W : S->workers) {
    if (W.stream) cudaStreamSynchronize(W.stream);
    if (W.ctx) fmm_destroy(W.ctx);
    if (W.stream) cudaStreamDestroy(W.stream);
    if (W.digest) cudaFree(W.digest);
  }
  for (auto& y : S->systems)
    if (y.xyz) cudaFree(y.xyz);
  cudaSetDevice(prev);
  delete S;
  return FMM_OK;
}

int fmm_server_add_system(fmm_server* S, const float* xyz, uint32_t n, int host, int L,
                          float sigma_scale, uint64_t seed, uint32_t* system) {
  if (!S || !system || (n > 0 && !xyz)) return FMM_ERR_ARG;
  if (L < 0 || L > kMaxLevel) return FMM_ERR_LEVEL;
  if (!(sigma_scale >= 0.f)) return FMM_ERR_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  System y;
  y.n = n;
  y.L = L;
  y.sigma = sigma_scale * std::ldexp(1.0f, -L);
  y.seed = seed;
  // workspace estimate of one build: sort buffers, boxes and lists per point
  y.est = 192ull * n + (4ull << 20);
  int st = FMM_OK;
  uint32_t* bad = nullptr;
  uint32_t hbad = 0;
  if (cudaMalloc(&y.xyz, sizeof(float) * 3 * std::max<uint32_t>(n, 1)) != cudaSuccess ||
      cudaMalloc(&bad, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(bad, 0, sizeof(uint32_t)) != cudaSuccess ||
      (n > 0 && cudaMemcpy(y.xyz, xyz, sizeof(float) * 3 * n,
                           host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice) !=
                    cudaSuccess)) {
    st = FMM_ERR_CUDA;
  } else if (n > 0) {
    const uint64_t cnt = 3ull * n;
    check_unit_kernel<<<(uint32_t)std::min<uint64_t>((cnt + 255) / 256, 152u * 8u), 256>>>(
        y.xyz, cnt, bad);
    if (cudaMemcpy(&hbad, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = FMM_ERR_CUDA;
    else if (hbad)
      st = FMM_ERR_DOMAIN;
  }
  if (bad) cudaFree(bad);
  if (st != FMM_OK) {
    cudaGetLastError();
    if (y.xyz) cudaFree(y.xyz);
    cudaSetDevice(prev);
    return st;
  }
  cudaSetDevice(prev);
  std::lock_guard<std::mutex> lk(S->mu);
  *system = (uint32_t)S->systems.size();
  S->systems.push_back(std::move(y));
  return FMM_OK;
}

int fmm_server_submit(fmm_server* S, uint32_t system, uint64_t* request_id) {
  if (!S || !request_id) return FMM_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (system >= S->systems.size() || S->stop) return FMM_ERR_ARG;
    *request_id = enqueue(S, system, now_s(S));
  }
  S->work_cv.notify_all();
  return FMM_OK;
}

int fmm_server_wait(fmm_server* S, uint64_t id, fmm_request_info* info) {
  if (!S) return FMM_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (id >= S->reqs.size()) return FMM_ERR_ARG;
  S->done_cv.wait(lk, [&] { return S->reqs[id]->done; });
  if (info) *info = S->reqs[id]->info;
  return (int)S->reqs[id]->info.status;
}

int fmm_server_poll(fmm_server* S, uint64_t id, fmm_request_info* info) {
  if (!S) return FMM_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (id >= S->reqs.size()) return FMM_ERR_ARG;
  if (!S->reqs[id]->done) return FMM_PENDING;
  if (info) *info = S->reqs[id]->info;
  return (int)S->reqs[id]->info.status;
}

int fmm_server_run_trace(fmm_server* S, const double* arrival_s, const uint32_t* system,
                         uint32_t count, fmm_request_info* info) {
  if (!S || (count > 0 && (!arrival_s || !system || !info))) return FMM_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (uint32_t k = 0; k < count; ++k)
      if (system[k] >= S->systems.size() || (k > 0 && arrival_s[k] < arrival_s[k - 1]))
        return FMM_ERR_ARG;
  }
  std::vector<uint64_t> ids(count);
  const double base = now_s(S);
  for (uint32_t k = 0; k < count; ++k) {
    const double t = base + arrival_s[k];
    const double wait = t - now_s(S);
    if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
    {
      std::lock_guard<std::mutex> lk(S->mu);
      ids[k] = enqueue(S, system[k], t);  // latency counts from the scheduled arrival
    }
    S->work_cv.notify_all();
  }
  int st = FMM_OK;
  std::unique_lock<std::mutex> lk(S->mu);
  for (uint32_t k = 0; k < count; ++k) {
    S->done_cv.wait(lk, [&] { return S->reqs[ids[k]]->done; });
    info[k] = S->reqs[ids[k]]->info;
    if (info[k].status != FMM_OK && st == FMM_OK) st = (int)info[k].status;
  }
  return st;
}

int fmm_server_points(fmm_server* S, uint32_t system, float* host_xyz) {
  if (!S || !host_xyz) return FMM_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (system >= S->systems.size()) return FMM_ERR_ARG;
  const System& y = S->systems[system];
  if (y.busy || !y.queue.empty()) return FMM_ERR_ARG;
  if (y.n == 0) return FMM_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  const cudaError_t e =
      cudaMemcpy(host_xyz, y.xyz, sizeof(float) * 3 * y.n, cudaMemcpyDeviceToHost);
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  return FMM_OK;
}

int fmm_server_tree(fmm_server* S, uint32_t system, fmm_tree* out) {
  if (!S || !out) return FMM_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (system >= S->systems.size()) return FMM_ERR_ARG;
  const System& y = S->systems[system];
  if (!y.has_last || y.busy || !y.queue.empty()) return FMM_ERR_ARG;
  if (S->workers[y.last_worker].gen == y.last_gen) {
    *out = y.last;  // still in the arena of the worker that built it
    return FMM_OK;
  }
  // That worker has built another batch since: build the same points again
  // (a build is a function of the points and L alone).
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  int st = FMM_OK;
  if (!S->qctx) {
    st = fmm_create(&S->qctx, S->device, nullptr, nullptr, nullptr);
    if (st == FMM_OK && cudaStreamCreateWithFlags(&S->qstream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      fmm_destroy(S->qctx);
      S->qctx = nullptr;
      st = FMM_ERR_CUDA;
    }
  }
  if (st == FMM_OK) {
    fmm_params p{y.L, 0, 0, 0};
    st = fmm_build(S->qctx, y.xyz, y.n, y.xyz, y.n, p, out, S->qstream);
  }
  cudaSetDevice(prev);
  return st;
}

}  // extern "C"
