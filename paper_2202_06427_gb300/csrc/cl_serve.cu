// cl_serve.cu -- continuous-batching request server (cellmap_serve.h).
//
// Device side: one persistent sweep kernel per batch. Its CTAs take work
// items from a device counter; item k of the batch is tile (k - base_r) of
// the request r whose item range holds k (a tile = 256 cell-sorted particles
// of one request). Each request carries its own geometry, stencil, cell list
// and outputs in a descriptor, so requests of different sizes, boxes,
// dimensions and tasks share one launch. A finalize kernel (one CTA per
// request) sums the per-tile FP64 partials in a fixed order.
//
// Host side: a scheduling thread admits requests by device-arena space,
// builds their cell lists on build streams, launches batches on the main
// stream (at most two in flight) and completes requests when their batch's
// event has fired.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cellmap_serve.h"
#include "cl_sweep.cuh"

namespace clk {

struct ReqDesc {
  int dim, task, n, noff;
  int nx, ny, nz, nbins;
  float rc2, irc, irc2, hscale, rmax;
  float ex, ey, ez;  // a cell's bounding-box half-widths (as in SweepArgs)
  int item_base, nitems;
  const float4* xs;
  const unsigned* cellc;
  const int* cell_start;
  const Off* off;
  float* forces;
  unsigned long long* hist;
  double* partials;
  double* energy;
  double* virial;
};

constexpr int kServeThreads = 256;

// One tile of a request: one thread per cell-sorted particle over the
// stencil, the packed (f32x2) sweep in 3D as in the library's per-particle
// kernels, the scalar one in 2D.
template <int DIM>
__device__ void serve_tile(const ReqDesc& R, int blk, unsigned* shist) {
  const int p = blk * kServeThreads + threadIdx.x;
  float4 pi;
  if (R.task == CL_TASK_ENERGY) {
    double v[1];
    if (DIM == 3) {
      Red2Energy red;
      red.irc = R.irc;
      Red2Energy::Acc acc;
      red.init(acc);
      sweep_particle2(R, red, acc, p, pi);
      v[0] = (double)acc.e.x + (double)acc.e.y;
    } else {
      RedEnergy red;
      red.irc = R.irc;
      RedEnergy::Acc acc;
      red.init(acc);
      sweep_particle<DIM>(R, red, acc, p, pi);
      v[0] = (double)acc.e;
    }
    block_sum_store<1>(v, R.partials + blk);
  } else if (R.task == CL_TASK_FORCES) {
    constexpr int NW = DIM == 3 ? 6 : 3;
    double v[NW + 1];
    if (DIM == 3) {
      Red2Force<true> red;
      red.irc = R.irc;
      red.irc2 = R.irc2;
      Red2Force<true>::Acc acc;
      red.init(acc);
      const bool live = sweep_particle2(R, red, acc, p, pi);
      float v6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (live) {
        const int i = __float_as_int(pi.w);
        R.forces[(size_t)i * 3 + 0] = -acc.tx;
        R.forces[(size_t)i * 3 + 1] = -acc.ty;
        R.forces[(size_t)i * 3 + 2] = -acc.tz;
        red.virial(acc, pi.x, pi.y, pi.z, v6);
      }
      // the scalar sweep's accumulator is sum fs r (x) r = -(sum fsn r (x) r)
      for (int k = 0; k < 6; ++k) v[k] = -(double)v6[k];
      v[NW] = 0.5 * ((double)acc.e.x + (double)acc.e.y);
    } else {
      RedForce<DIM, true> red;
      red.irc = R.irc;
      red.irc2 = R.irc2;
      typename RedForce<DIM, true>::Acc acc;
      red.init(acc);
      const bool live = sweep_particle<DIM>(R, red, acc, p, pi);
      if (live) {
        const int i = __float_as_int(pi.w);
#pragma unroll
        for (int a = 0; a < DIM; ++a) R.forces[(size_t)i * DIM + a] = acc.f[a];
      }
      v[0] = acc.w[0]; v[1] = acc.w[1]; v[2] = acc.w[3];
      v[NW] = 0.5 * (double)acc.e;
    }
    block_sum_store<NW + 1>(v, R.partials + (size_t)blk * (NW + 1));
  } else {
    for (int b = threadIdx.x; b < R.nbins; b += blockDim.x) shist[b] = 0u;
    __syncthreads();
    if (DIM == 3) {
      Red2Hist red;
      red.scale2 = R.hscale * R.hscale;
      red.xlim = fminf((float)R.nbins, sqrtf(R.rc2) * R.hscale);
      red.sh = shist;
      Red2Hist::Acc acc;
      sweep_particle2(R, red, acc, p, pi);
    } else {
      RedHist red;
      red.nbins = R.nbins;
      red.rmax = R.rmax;
      red.scale = R.hscale;
      red.sh = shist;
      RedHist::Acc acc;
      sweep_particle<DIM>(R, red, acc, p, pi);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < R.nbins; b += blockDim.x)
      if (shist[b]) atomicAdd(&R.hist[b], (unsigned long long)shist[b]);
  }
}

__global__ void __launch_bounds__(kServeThreads) k_serve_sweep(const ReqDesc* __restrict__ reqs, int nreq,
                                                                int nitems, int* __restrict__ counter) {
  extern __shared__ unsigned shist[];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    int lo = 0, hi = nreq - 1;  // last request whose item range starts at or before it
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (reqs[mid].item_base <= it) lo = mid;
      else hi = mid - 1;
    }
    const ReqDesc R = reqs[lo];
    const int blk = it - R.item_base;
    if (R.dim == 3) serve_tile<3>(R, blk, shist);
    else serve_tile<2>(R, blk, shist);
  }
}

// One CTA per request: fixed-order FP64 sums of the tile partials.
__global__ void __launch_bounds__(256) k_serve_finalize(const ReqDesc* __restrict__ reqs) {
  const ReqDesc R = reqs[blockIdx.x];
  if (R.task == CL_TASK_HIST) return;
  const int d = R.dim;
  const int NW = d == 3 ? 6 : 3;
  const int nv = R.task == CL_TASK_ENERGY ? 1 : NW + 1;
  __shared__ double sm[256];
  __shared__ double sums[8];
  for (int k = 0; k < nv; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < R.nitems; b += 256) s += R.partials[(size_t)b * nv + k];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) sums[k] = sm[0];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  if (R.task == CL_TASK_ENERGY) {
    *R.energy = sums[0];
    return;
  }
  *R.energy = sums[NW];
  double S[3][3];
  if (d == 3) {
    const int map[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) S[a][b] = sums[map[a][b]];
  } else {
    S[0][0] = sums[0]; S[0][1] = S[1][0] = sums[1]; S[1][1] = sums[2];
  }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) R.virial[a * d + b] = -0.5 * S[a][b];
}

}  // namespace clk

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kBuildStreams = 4;
constexpr size_t kAlign = 256;
// Requests admitted per pass of the scheduling loop before it looks for a free
// batch slot: admission (copies and binning launches, about a dozen runtime
// calls per request) is host work, and a burst of hundreds of requests
// admitted in one pass would keep the GPU waiting for the first batch.
constexpr int kAdmitPerPass = 32;

size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over the device arena, with coalescing of free blocks.
class Arena {
 public:
  void init(size_t bytes) {
    size_ = bytes;
    free_.clear();
    free_[0] = bytes;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t size() const { return size_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0;
};

struct Req {
  cl_request r;
  long long ticket;
  int status = 1;
  double t[4] = {0, 0, 0, 0};
  clk::Geo geo;
  std::vector<clk::Off> off;
  size_t arena_off = 0, arena_bytes = 0;
  clk::BuildBufs bufs;
  clk::Off* d_off = nullptr;
  float* d_forces = nullptr;
  unsigned long long* d_hist = nullptr;
  double* d_partials = nullptr;
  double* d_energy = nullptr;
  double* d_virial = nullptr;
  int latched = 0;  // host copy of the error latch
  int nitems = 0;
  cudaEvent_t built = nullptr;
};

struct Batch {
  std::vector<Req*> reqs;
  clk::ReqDesc* h_desc = nullptr;  // pinned
  clk::ReqDesc* d_desc = nullptr;
  int* d_counter = nullptr;
  int* h_latch = nullptr;          // pinned, one per request of the batch
  cudaEvent_t done = nullptr;
  bool busy = false;
  int err = CL_OK;                 // CL_ERR_CUDA when a copy or launch of the batch failed
};

}  // namespace

struct cl_server {
  int device = 0;
  int max_inflight = 0;
  cudaStream_t main = nullptr;
  cudaStream_t build[kBuildStreams] = {};
  int next_build = 0;
  char* arena_base = nullptr;
  Arena arena;
  Batch batches[2];
  int sm_count = 0;
  int ctas_per_sm = 0;
  Clock::time_point t0;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  long long next_ticket = 1;
  std::deque<Req*> incoming;  // submitted, not yet seen by the thread (under mu)
  std::deque<Req*> queue;     // waiting for admission (thread only)
  std::vector<Req*> ready;    // admitted, not yet in a batch (thread only)
  int resident = 0;           // admitted and not completed (thread only)
  std::unordered_map<long long, Req*> all;  // under mu
  long long stats[6] = {0, 0, 0, 0, 0, 0};  // under mu

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void loop();
  bool admit_one(Req* q);
  void launch_batch(Batch& b);
  void complete(Batch& b);
  void finish(Req* q, int status);
};

namespace {

// Device bytes a request needs: positions, binning buffers, cell offsets,
// stencil, partials and outputs, each piece 256-byte aligned.
size_t request_bytes(const Req& q) {
  const size_t n = (size_t)q.r.n, d = (size_t)q.geo.dim, C = (size_t)q.geo.ncells;
  const size_t tiles = (size_t)clk::scan_tiles_for((long long)C);
  const size_t items = n > 0 ? (n + clk::kServeThreads - 1) / clk::kServeThreads : 1;
  size_t b = up(n * d * 8) + 2 * up(n * 16) + 2 * up(n * 4) + up(C * 4) + up((C + 1) * 4) + up(tiles * 4 + 4) +
             up(16) + up(q.off.size() * sizeof(clk::Off)) + up(items * 7 * 8) + up(8) + up(72);
  if (q.r.task == CL_TASK_FORCES) b += up(n * d * 4);
  if (q.r.task == CL_TASK_HIST) b += up((size_t)q.r.nbins * 8);
  return b;
}

}  // namespace

void cl_server::finish(Req* q, int status) {
  // the request's work is over: its event and stencil copy are no longer
  // needed, only the status and timestamps stay until the ticket is released
  if (q->built) {
    cudaEventDestroy(q->built);
    q->built = nullptr;
  }
  std::vector<clk::Off>().swap(q->off);
  {
    std::lock_guard<std::mutex> g(mu);
    q->status = status;
    q->t[3] = now();
    if (status == 0) stats[1]++;
    else stats[2]++;
    stats[4] = (long long)arena.used();  // finish() runs on the scheduling thread, which owns the arena
  }
  cv_done.notify_all();
}

bool cl_server::admit_one(Req* q) {
  const size_t bytes = request_bytes(*q);
  if (bytes > arena.size()) {
    finish(q, CL_ERR_OOM);
    return true;
  }
  size_t off;
  if (!arena.alloc(bytes, &off)) return false;
  q->arena_off = off;
  q->arena_bytes = bytes;
  char* p = arena_base + off;
  auto take = [&](size_t sz) {
    char* r = p;
    p += up(sz);
    return r;
  };
  const size_t n = (size_t)q->r.n, d = (size_t)q->geo.dim, C = (size_t)q->geo.ncells;
  clk::BuildBufs& B = q->bufs;
  B.pos = reinterpret_cast<const double*>(take(n * d * 8));
  B.n = (int)n;
  B.xl = reinterpret_cast<float4*>(take(n * 16));
  B.xs = reinterpret_cast<float4*>(take(n * 16));
  B.slot = reinterpret_cast<int*>(take(n * 4));
  B.cellc = reinterpret_cast<unsigned*>(take(n * 4));
  B.counts = reinterpret_cast<int*>(take(C * 4));
  B.cell_start = reinterpret_cast<int*>(take((C + 1) * 4));
  B.tile_sum = reinterpret_cast<int*>(take((size_t)clk::scan_tiles_for((long long)C) * 4 + 4));
  B.meta = reinterpret_cast<int*>(take(16));
  q->d_off = reinterpret_cast<clk::Off*>(take(q->off.size() * sizeof(clk::Off)));
  q->nitems = n > 0 ? (int)((n + clk::kServeThreads - 1) / clk::kServeThreads) : 0;
  q->d_partials = reinterpret_cast<double*>(take((size_t)std::max(q->nitems, 1) * 7 * 8));
  q->d_energy = reinterpret_cast<double*>(take(8));
  q->d_virial = reinterpret_cast<double*>(take(72));
  if (q->r.task == CL_TASK_FORCES) q->d_forces = reinterpret_cast<float*>(take(n * d * 4));
  if (q->r.task == CL_TASK_HIST) q->d_hist = reinterpret_cast<unsigned long long*>(take((size_t)q->r.nbins * 8));
  cudaStream_t s = build[next_build];
  next_build = (next_build + 1) % kBuildStreams;
  int e = CL_OK;
  if (n > 0 && cudaMemcpyAsync((void*)B.pos, q->r.pos_host, n * d * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
    e = CL_ERR_CUDA;
  if (!e && cudaMemcpyAsync(q->d_off, q->off.data(), q->off.size() * sizeof(clk::Off), cudaMemcpyHostToDevice, s) !=
                cudaSuccess)
    e = CL_ERR_CUDA;
  if (!e && cudaMemsetAsync(B.meta, 0, 16, s) != cudaSuccess) e = CL_ERR_CUDA;
  if (!e && q->d_hist && cudaMemsetAsync(q->d_hist, 0, (size_t)q->r.nbins * 8, s) != cudaSuccess) e = CL_ERR_CUDA;
  if (!e && cudaMemsetAsync(q->d_energy, 0, 8 + 72, s) != cudaSuccess) e = CL_ERR_CUDA;
  if (!e) e = clk::launch_build(q->geo, B, s);
  if (!e && cudaEventRecord(q->built, s) != cudaSuccess) e = CL_ERR_CUDA;
  {
    std::lock_guard<std::mutex> g(mu);
    q->t[1] = now();
  }
  if (e) {
    cudaStreamSynchronize(s);
    arena.release(q->arena_off, q->arena_bytes);
    finish(q, e);
    return true;
  }
  resident++;
  ready.push_back(q);
  return true;
}

void cl_server::launch_batch(Batch& b) {
  b.reqs.swap(ready);
  ready.clear();
  b.err = CL_OK;
  // every enqueue is checked; after the first failure nothing more is
  // launched and complete() fails the batch's requests with CL_ERR_CUDA
  auto ok = [&b](cudaError_t r) {
    if (r != cudaSuccess && !b.err) b.err = CL_ERR_CUDA;
  };
  int items = 0, maxbins = 0;
  const double tl = now();
  for (size_t k = 0; k < b.reqs.size(); ++k) {
    Req* q = b.reqs[k];
    q->t[2] = tl;
    clk::ReqDesc& D = b.h_desc[k];
    std::memset(&D, 0, sizeof(D));
    D.dim = q->geo.dim;
    D.task = q->r.task;
    D.n = (int)q->r.n;
    D.noff = (int)q->off.size();
    D.nx = q->geo.n[0];
    D.ny = q->geo.n[1];
    D.nz = q->geo.n[2];
    D.nbins = q->r.nbins;
    D.rc2 = (float)(q->geo.rc * q->geo.rc);
    D.irc = (float)(1.0 / q->geo.rc);
    D.irc2 = (float)(1.0 / (q->geo.rc * q->geo.rc));
    {
      float e[3];
      clk::cell_halfwidths(q->geo, e);
      D.ex = e[0];
      D.ey = e[1];
      D.ez = e[2];
    }
    const double rmax = q->r.rmax > 0 ? q->r.rmax : q->geo.rc;
    D.rmax = (float)rmax;
    D.hscale = q->r.task == CL_TASK_HIST ? (float)(q->r.nbins / rmax) : 0.f;
    D.item_base = items;
    D.nitems = q->nitems;
    D.xs = q->bufs.xs;
    D.cellc = q->bufs.cellc;
    D.cell_start = q->bufs.cell_start;
    D.off = q->d_off;
    D.forces = q->d_forces;
    D.hist = q->d_hist;
    D.partials = q->d_partials;
    D.energy = q->d_energy;
    D.virial = q->d_virial;
    items += q->nitems;
    if (q->r.task == CL_TASK_HIST) maxbins = std::max(maxbins, q->r.nbins);
    ok(cudaStreamWaitEvent(main, q->built, 0));
  }
  const int nreq = (int)b.reqs.size();
  ok(cudaMemcpyAsync(b.d_desc, b.h_desc, sizeof(clk::ReqDesc) * nreq, cudaMemcpyHostToDevice, main));
  ok(cudaMemsetAsync(b.d_counter, 0, sizeof(int), main));
  if (items > 0 && !b.err) {
    int grid = std::min(items, sm_count * ctas_per_sm);
    clk::k_serve_sweep<<<grid, clk::kServeThreads, sizeof(unsigned) * maxbins, main>>>(b.d_desc, nreq, items,
                                                                                       b.d_counter);
    ok(cudaGetLastError());
  }
  if (!b.err) {
    clk::k_serve_finalize<<<nreq, 256, 0, main>>>(b.d_desc);
    ok(cudaGetLastError());
  }
  for (int k = 0; k < nreq && !b.err; ++k) {
    Req* q = b.reqs[k];
    const size_t n = (size_t)q->r.n, d = (size_t)q->geo.dim;
    if (q->r.task != CL_TASK_HIST && q->r.energy_host)
      ok(cudaMemcpyAsync(q->r.energy_host, q->d_energy, 8, cudaMemcpyDeviceToHost, main));
    if (q->r.task == CL_TASK_FORCES) {
      if (q->r.forces_host && n)
        ok(cudaMemcpyAsync(q->r.forces_host, q->d_forces, n * d * 4, cudaMemcpyDeviceToHost, main));
      if (q->r.virial_host)
        ok(cudaMemcpyAsync(q->r.virial_host, q->d_virial, d * d * 8, cudaMemcpyDeviceToHost, main));
    }
    if (q->r.task == CL_TASK_HIST && q->r.hist_host)
      ok(cudaMemcpyAsync(q->r.hist_host, q->d_hist, (size_t)q->r.nbins * 8, cudaMemcpyDeviceToHost, main));
    ok(cudaMemcpyAsync(b.h_latch + k, q->bufs.meta, sizeof(int), cudaMemcpyDeviceToHost, main));
  }
  if (cudaEventRecord(b.done, main) != cudaSuccess) {
    // no event to poll: wait for what was queued, then finish the batch now
    b.err = CL_ERR_CUDA;
    cudaStreamSynchronize(main);
    b.busy = true;
    complete(b);
  } else {
    b.busy = true;
  }
  std::lock_guard<std::mutex> g(mu);
  stats[0]++;
  stats[3] = std::max<long long>(stats[3], nreq);
}

void cl_server::complete(Batch& b) {
  for (size_t k = 0; k < b.reqs.size(); ++k) {
    Req* q = b.reqs[k];
    arena.release(q->arena_off, q->arena_bytes);
    resident--;
    finish(q, b.err ? b.err : (b.h_latch[k] & clk::kErrNonFinite) ? CL_ERR_NONFINITE : 0);
  }
  b.reqs.clear();
  b.busy = false;
  b.err = CL_OK;
}

void cl_server::loop() {
  cudaSetDevice(device);
  for (;;) {
    bool progressed = false;
    {
      std::unique_lock<std::mutex> g(mu);
      while (!incoming.empty()) {
        queue.push_back(incoming.front());
        incoming.pop_front();
      }
      const bool idle = queue.empty() && ready.empty() && !batches[0].busy && !batches[1].busy;
      if (idle) {
        if (stop) break;
        cv_work.wait_for(g, std::chrono::milliseconds(2));
        continue;
      }
    }
    // completions first: they free arena space for admission
    for (Batch& b : batches)
      if (b.busy && cudaEventQuery(b.done) == cudaSuccess) {
        complete(b);
        progressed = true;
      }
    for (int k = 0; k < kAdmitPerPass && !queue.empty() && resident < max_inflight; ++k) {
      Req* q = queue.front();
      if (!admit_one(q)) break;
      queue.pop_front();
      progressed = true;
    }
    if (!ready.empty())
      for (Batch& b : batches)
        if (!b.busy) {
          launch_batch(b);
          progressed = true;
          break;
        }
    {
      std::lock_guard<std::mutex> g(mu);
      stats[4] = (long long)arena.used();
    }
    if (!progressed) std::this_thread::yield();
  }
}

extern "C" {

int cl_serve_create(long long arena_bytes, int max_inflight, int device, cl_server** out) {
  if (!out || arena_bytes <= 0 || max_inflight < 1 || max_inflight > 1024) return CL_ERR_INVALID_ARG;
  *out = nullptr;
  cl_server* s = new (std::nothrow) cl_server;
  if (!s) return CL_ERR_OOM;
  s->device = device;
  s->max_inflight = max_inflight;
  s->t0 = Clock::now();
  int e = CL_OK;
  if (cudaSetDevice(device) != cudaSuccess) e = CL_ERR_CUDA;
  cudaDeviceProp prop;
  if (!e && cudaGetDeviceProperties(&prop, device) != cudaSuccess) e = CL_ERR_CUDA;
  if (!e) {
    s->sm_count = prop.multiProcessorCount;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, clk::k_serve_sweep, clk::kServeThreads,
                                                      sizeof(unsigned) * clk::kMaxBins) != cudaSuccess)
      e = CL_ERR_CUDA;
    s->ctas_per_sm = std::max(per, 1);
  }
  if (!e && cudaMalloc((void**)&s->arena_base, (size_t)arena_bytes) != cudaSuccess) e = CL_ERR_OOM;
  if (!e) s->arena.init((size_t)arena_bytes);
  if (!e && cudaStreamCreateWithFlags(&s->main, cudaStreamNonBlocking) != cudaSuccess) e = CL_ERR_CUDA;
  for (int k = 0; k < kBuildStreams && !e; ++k)
    if (cudaStreamCreateWithFlags(&s->build[k], cudaStreamNonBlocking) != cudaSuccess) e = CL_ERR_CUDA;
  for (Batch& b : s->batches) {
    if (e) break;
    if (cudaMallocHost((void**)&b.h_desc, sizeof(clk::ReqDesc) * max_inflight) != cudaSuccess ||
        cudaMalloc((void**)&b.d_desc, sizeof(clk::ReqDesc) * max_inflight) != cudaSuccess ||
        cudaMalloc((void**)&b.d_counter, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&b.h_latch, sizeof(int) * max_inflight) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess)
      e = CL_ERR_OOM;
  }
  if (e) {
    cl_serve_free(s);
    return e;
  }
  s->th = std::thread([s] { s->loop(); });
  *out = s;
  return CL_OK;
}

int cl_serve_submit(cl_server* s, const cl_request* req, long long* ticket) {
  if (!s || !req || !ticket || req->n < 0 || req->n >= 2147483647LL || (req->n > 0 && !req->pos_host))
    return CL_ERR_INVALID_ARG;
  if (req->task < CL_TASK_ENERGY || req->task > CL_TASK_HIST) return CL_ERR_INVALID_ARG;
  if (req->task == CL_TASK_HIST && (req->nbins < 1 || req->nbins > clk::kMaxBins || !req->hist_host))
    return CL_ERR_INVALID_ARG;
  if (req->task == CL_TASK_FORCES && req->n > 0 && !req->forces_host) return CL_ERR_INVALID_ARG;
  Req* q = new (std::nothrow) Req;
  if (!q) return CL_ERR_OOM;
  q->r = *req;
  int e = clk::prepare_geometry(&req->box, &q->geo);
  if (!e) {
    q->off.resize(clk::kMaxOff);
    int noff = clk::build_stencil(q->geo, req->task == CL_TASK_FORCES ? 0 : 1, q->off.data(), clk::kMaxOff);
    if (noff < 0) e = noff;
    else q->off.resize(noff);
  }
  if (!e && cudaEventCreateWithFlags(&q->built, cudaEventDisableTiming) != cudaSuccess) e = CL_ERR_CUDA;
  if (e) {
    delete q;
    return e;
  }
  {
    std::lock_guard<std::mutex> g(s->mu);
    q->ticket = s->next_ticket++;
    q->t[0] = s->now();
    s->all[q->ticket] = q;
    s->incoming.push_back(q);
    *ticket = q->ticket;
  }
  s->cv_work.notify_one();
  return CL_OK;
}

int cl_serve_poll(cl_server* s, long long ticket) {
  if (!s) return CL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->all.find(ticket);
  return it == s->all.end() ? CL_ERR_INVALID_ARG : it->second->status;
}

int cl_serve_wait(cl_server* s, long long ticket, double timeout_s) {
  if (!s) return CL_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> g(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return CL_ERR_INVALID_ARG;
  Req* q = it->second;
  s->cv_done.wait_for(g, std::chrono::duration<double>(timeout_s), [q] { return q->status != 1; });
  return q->status;
}

int cl_serve_times(cl_server* s, long long ticket, double* times) {
  if (!s || !times) return CL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return CL_ERR_INVALID_ARG;
  for (int k = 0; k < 4; ++k) times[k] = it->second->t[k];
  return CL_OK;
}

int cl_serve_stats(cl_server* s, long long* out) {
  if (!s || !out) return CL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  for (int k = 0; k < 5; ++k) out[k] = s->stats[k];
  out[5] = (long long)s->arena.size();
  return CL_OK;
}

double cl_serve_clock(cl_server* s) { return s ? s->now() : 0.0; }

int cl_serve_release(cl_server* s, long long ticket) {
  if (!s) return CL_ERR_INVALID_ARG;
  Req* q = nullptr;
  {
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return CL_ERR_INVALID_ARG;
    if (it->second->status == 1) return 1;  // still pending: kept
    q = it->second;
    s->all.erase(it);
  }
  delete q;  // finish() already destroyed its event
  return CL_OK;
}

void cl_serve_free(cl_server* s) {
  if (!s) return;
  if (s->th.joinable()) {
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    s->th.join();
  }
  cudaSetDevice(s->device);
  if (s->main) cudaStreamSynchronize(s->main);
  for (int k = 0; k < kBuildStreams; ++k)
    if (s->build[k]) {
      cudaStreamSynchronize(s->build[k]);
      cudaStreamDestroy(s->build[k]);
    }
  if (s->main) cudaStreamDestroy(s->main);
  for (Batch& b : s->batches) {
    cudaFreeHost(b.h_desc);
    cudaFree(b.d_desc);
    cudaFree(b.d_counter);
    cudaFreeHost(b.h_latch);
    if (b.done) cudaEventDestroy(b.done);
  }
  cudaFree(s->arena_base);
  for (auto& kv : s->all) {
    if (kv.second->built) cudaEventDestroy(kv.second->built);
    delete kv.second;
  }
  delete s;
}

}  // extern "C"
