// sort_static.cu -- cell sort of caller-owned particle arrays that allocates
// nothing.
//
// pic1d_sort (through a context) keeps its histogram, offsets and block sums
// in memory the context obtained from cudaMalloc.  Some callers cannot
// allocate device memory at all: code running inside a memory pool they do
// not control, or on a device whose memory is fully reserved up front.  For
// them this file holds the same scratch in one file-scope device array of
// fixed size, which every GPU that loads the library keeps until the process
// exits, and runs the same sort kernels on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "pic1d_internal.h"

using namespace pic1d;

namespace {

constexpr int kStaticMaxCells = PIC1D_SORT_STATIC_MAX_CELLS;
constexpr int kStaticBins = 4 * kSortBands * kStaticMaxCells;   // key = ((2 ion + (u < 0)) n_cells + cell) kSortBands + band
constexpr int kStaticChunk = 4096;                         // bins per scan block
constexpr size_t kCountsBytes = sizeof(uint32_t) * kStaticBins;
constexpr size_t kOffsetsBytes = sizeof(long long) * (kStaticBins + 1);
constexpr size_t kBsumBytes = sizeof(long long) * ((kStaticBins + kStaticChunk - 1) / kStaticChunk);
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffCounts = 0;
constexpr size_t kOffOffsets = align_up(kOffCounts + kCountsBytes);
constexpr size_t kOffBsum = align_up(kOffOffsets + kOffsetsBytes);
constexpr size_t kOffState = align_up(kOffBsum + kBsumBytes);
constexpr size_t kScratchBytes = align_up(kOffState + sizeof(StepState));

// The scratch: histogram | offsets | block sums | slot counters.  In host code
// the name is only a stand-in for the device symbol; the device address comes
// from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

// device address of the scratch in the current context, looked up on every
// call (cheap, no stream work): a cached address would go stale when the
// context is reset and the module loaded again
cudaError_t scratch_on_current_device(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

__global__ void k_static_begin(StepState* st, long long n) {
  st->n_slots = n;
  st->append = 0;
  st->sorted_total = 0;
}

__global__ void k_static_end(const StepState* st, long long* n_out) { *n_out = st->sorted_total; }

int fbits_for(int n) {
  int b = 0;
  while ((1 << b) < n) ++b;
  return 32 - b;
}

}  // namespace

extern "C" int pic1d_sort_static(int32_t n_cells, int64_t n, const uint32_t* pos, const float* u, const float* w,
                                 const uint8_t* sp, const uint64_t* id, uint32_t* pos_out, float* u_out,
                                 float* w_out, uint8_t* sp_out, uint64_t* id_out, int64_t* n_out,
                                 void* cuda_stream) {
  if (n_cells < 8 || n_cells > kStaticMaxCells) {
    std::fprintf(stderr, "pic1d_sort_static: n_cells = %d outside [8, %d] (the static scratch is sized for %d cells)\n",
                 n_cells, kStaticMaxCells, kStaticMaxCells);
    return PIC1D_EINVAL;
  }
  if (n < 0 || n >= (1ll << 31) || !n_out ||
      (n > 0 && (!pos || !u || !w || !sp || !id || !pos_out || !u_out || !w_out || !sp_out || !id_out))) {
    std::fprintf(stderr, "pic1d_sort_static: bad arguments\n");
    return PIC1D_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  unsigned char* base = nullptr;
  cudaError_t e = scratch_on_current_device(&base);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "pic1d_sort_static: scratch address: %s\n", cudaGetErrorString(e));
    return PIC1D_ECUDA;
  }
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "pic1d_sort_static: %s\n", cudaGetErrorString(e));
    return PIC1D_ECUDA;
  }
  uint32_t* counts = reinterpret_cast<uint32_t*>(base + kOffCounts);
  long long* offsets = reinterpret_cast<long long*>(base + kOffOffsets);
  long long* bsum = reinterpret_cast<long long*>(base + kOffBsum);
  StepState* st = reinterpret_cast<StepState*>(base + kOffState);

  DevParams P{};
  P.N = n_cells;
  P.F = fbits_for(n_cells);
  P.top = (long long)n_cells << P.F;
  P.pos = const_cast<uint32_t*>(pos);
  P.u = const_cast<float*>(u);
  P.w = const_cast<float*>(w);
  P.sp = const_cast<uint8_t*>(sp);
  P.id = const_cast<uint64_t*>(id);
  P.st = st;
  k_static_begin<<<1, 1, 0, s>>>(st, (long long)n);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = launch_sort(P, counts, offsets, bsum, pos_out, u_out, w_out, sp_out, id_out, std::max(1, sms), s);
  if (e == cudaSuccess) {
    k_static_end<<<1, 1, 0, s>>>(st, reinterpret_cast<long long*>(n_out));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    std::fprintf(stderr, "pic1d_sort_static: %s\n", cudaGetErrorString(e));
    return PIC1D_ECUDA;
  }
  return PIC1D_OK;
}
