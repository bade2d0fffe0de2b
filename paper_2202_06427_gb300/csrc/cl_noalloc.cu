// cl_noalloc.cu -- shifted-force energy of a small particle set without any
// device allocation (cl_energy_noalloc in cellmap.h).
//
// Who needs it: applications that hand all device memory to their own pool
// (a deep-learning framework's caching allocator, a simulation engine's fixed
// arena) and forbid raw cudaMalloc/cudaFree calls, and latency-critical loops
// where the synchronisation and cost of cudaMalloc are not acceptable. They
// cannot use cl_build, which allocates the cell-list workspace.
//
// Every buffer the binning and the energy sweep need (local coordinates,
// sorted particles, per-cell counts and offsets, per-CTA partial sums) lives
// in one file-scope __device__ array of fixed size, carved into 256-byte
// aligned pieces. Each GPU that loads the library holds this array
// (3,179,776 bytes) until the process exits. Host code only ever passes the
// array's device address, obtained once per device with cudaGetSymbolAddress;
// the host-side name of the array is a stand-in, never a device pointer.
//
// All calls share the array and it keeps the contents of the last call: the
// per-cell counts and the error word are cleared at the start of every call,
// everything else is fully rewritten before it is read. Calls whose GPU work
// overlaps (on different streams, or from different host threads without
// ordering) race on the array and give wrong results.
#include <atomic>

#include "cl_internal.cuh"

namespace {

constexpr long long kMaxN = CL_NOALLOC_MAX_N;
constexpr long long kMaxCells = CL_NOALLOC_MAX_CELLS;
constexpr int kMaxDevices = 64;

constexpr size_t up256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffXl = 0;
constexpr size_t kOffXs = kOffXl + up256(16 * kMaxN);
constexpr size_t kOffSlot = kOffXs + up256(16 * kMaxN);
constexpr size_t kOffCellc = kOffSlot + up256(4 * kMaxN);
constexpr size_t kOffCounts = kOffCellc + up256(4 * kMaxN);
constexpr size_t kOffStart = kOffCounts + up256(4 * kMaxCells);
constexpr size_t kOffTiles = kOffStart + up256(4 * (kMaxCells + 1));
constexpr size_t kOffMeta = kOffTiles + up256(4 * ((kMaxCells + 2047) / 2048 + 1));
constexpr size_t kOffPartials = kOffMeta + 256;
constexpr size_t kOffSums = kOffPartials + up256(8 * 16 * ((kMaxN + 255) / 256 + 1));
constexpr size_t kScratchBytes = kOffSums + 256;
static_assert(kScratchBytes == 3179776, "the workspace size stated in cellmap.h");

}  // namespace

static __device__ __align__(256) unsigned char g_cl_noalloc_scratch[kScratchBytes];

// Device address of the scratch array for the current device, looked up on the
// first call made with that device current and cached afterwards.
static std::atomic<unsigned char*> g_noalloc_ptr[kMaxDevices];

static int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CL_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return CL_ERR_UNSUPPORTED;
  unsigned char* p = g_noalloc_ptr[dev].load();
  if (p == nullptr) {
    void* q = nullptr;
    if (cudaGetSymbolAddress(&q, g_cl_noalloc_scratch) != cudaSuccess) return CL_ERR_CUDA;
    p = static_cast<unsigned char*>(q);
    g_noalloc_ptr[dev].store(p);
  }
  *out = p;
  return CL_OK;
}

// Half-shell stencil of the whole reach box (own cell first, then the
// lexicographically positive offsets), written in place without pruning: an
// offset whose cells are farther apart than rc simply finds no pair.
static int noalloc_stencil(const clk::Geo& g, clk::Off* out, int cap) {
  int m[3] = {0, 0, 0};
  for (int k = 0; k < g.dim; ++k) m[k] = (int)ceil(g.rc * g.n[k] / g.w[k]);
  int cnt = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int oz = -m[2]; oz <= m[2]; ++oz)
      for (int oy = -m[1]; oy <= m[1]; ++oy)
        for (int ox = -m[0]; ox <= m[0]; ++ox) {
          const bool self = (ox == 0 && oy == 0 && oz == 0);
          if ((pass == 0) != self) continue;
          if (!self && !((oz > 0) || (oz == 0 && (oy > 0 || (oy == 0 && ox > 0))))) continue;
          if (cnt == cap) return CL_ERR_UNSUPPORTED;
          const int o[3] = {ox, oy, oz};
          clk::Off e;
          int d[3];
          for (int k = 0; k < 3; ++k) d[k] = ((o[k] % g.n[k]) + g.n[k]) % g.n[k];
          e.dx = d[0];
          e.dy = d[1];
          e.dz = d[2];
          double s[3] = {0, 0, 0};
          for (int k = 0; k < g.dim; ++k)
            for (int a = 0; a < 3; ++a) s[a] += (double)o[k] / g.n[k] * g.h[k * 3 + a];
          e.sx = (float)s[0];
          e.sy = (float)s[1];
          e.sz = (float)s[2];
          out[cnt++] = e;
        }
  return cnt;
}

extern "C" int cl_energy_noalloc(const double* pos_dev, long long n, const cl_box* box, double* energy_dev,
                                 void* stream) {
  if (!box || !energy_dev || n < 0 || (n > 0 && !pos_dev)) return CL_ERR_INVALID_ARG;
  if (n > kMaxN) return CL_ERR_UNSUPPORTED;
  clk::Geo g;
  int e = clk::prepare_geometry(box, &g);
  if (e) return e;
  if (g.ncells > kMaxCells) return CL_ERR_UNSUPPORTED;
  clk::SweepArgs A;  // 18 KB of host-side launch arguments, on the stack
  const int noff = noalloc_stencil(g, A.off, clk::kMaxOff);
  if (noff < 0) return noff;
  unsigned char* base = nullptr;
  if ((e = noalloc_scratch(&base))) return e;
  cudaStream_t s = (cudaStream_t)stream;
  clk::BuildBufs b;
  b.pos = pos_dev;
  b.n = (int)n;
  b.xl = reinterpret_cast<float4*>(base + kOffXl);
  b.xs = reinterpret_cast<float4*>(base + kOffXs);
  b.slot = reinterpret_cast<int*>(base + kOffSlot);
  b.cellc = reinterpret_cast<unsigned*>(base + kOffCellc);
  b.counts = reinterpret_cast<int*>(base + kOffCounts);
  b.cell_start = reinterpret_cast<int*>(base + kOffStart);
  b.tile_sum = reinterpret_cast<int*>(base + kOffTiles);
  b.meta = reinterpret_cast<int*>(base + kOffMeta);
  if (cudaMemsetAsync(b.meta, 0, 4 * sizeof(int), s) != cudaSuccess) return CL_ERR_CUDA;
  if ((e = clk::launch_build(g, b, s))) return e;
  A.xs = b.xs;
  A.cellc = b.cellc;
  A.cell_start = b.cell_start;
  A.n = (int)n;
  A.nx = g.n[0];
  A.ny = g.n[1];
  A.nz = g.n[2];
  A.rc2 = (float)(g.rc * g.rc);
  A.irc = (float)(1.0 / g.rc);
  A.irc2 = (float)(1.0 / (g.rc * g.rc));
  A.ex = A.ey = A.ez = 0.f;  // the scalar sweep tests every stencil cell
  A.noff = noff;
  return clk::launch_scalar(A, g.dim, 1, reinterpret_cast<double*>(base + kOffPartials),
                            reinterpret_cast<double*>(base + kOffSums), energy_dev, s);
}
