// sort_noalloc.cu -- pic_sort_by_cell_noalloc: the (cell, id) sort of
// pic_sort_by_cell for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or cudaMallocAsync) where they need
// the sort: an application whose own memory pool has reserved the device up
// front, so that any other allocation fails; an embedder whose allocator must
// own every device byte; or a latency-bound loop that must not enter the
// driver's allocator, which can synchronise the device or fail under memory
// pressure.  This entry point takes the sort's scratch from a fixed array
// that is part of the library's device image instead.
//
// The array is a file-scope __device__ variable of kNoAllocScratchBytes
// (7,340,800 B: exactly the scratch of a sort at both limits below).  Under
// CUDA's lazy module loading (the default) a device gets the array when the
// library first asks for its address there, which this entry point does on
// its first call on that device: make that first call (n = 0 is enough)
// before the application reserves the device's memory for itself, and outside
// any stream capture.  From then on the device holds the array until the
// process exits.  Host code must not use the array's name as a device
// address: it is a host-side stand-in.  The address is looked up with
// cudaGetSymbolAddress on the current device on every call made outside a
// stream capture (this allocates nothing once the array is loaded, and stays
// right after a cudaDeviceReset); a call on a capturing stream uses the
// address cached by the device's last call outside capture.  All calls share
// the one array and it keeps the last call's contents, so calls whose work
// overlaps on the GPU (different streams, or host threads without ordering
// between them) race: order them.
#include <mutex>

#include "pic_internal.cuh"

namespace pic {

// Limits of the no-allocation sort, and the array sized for a call at both.
constexpr size_t kNoAllocMaxItems = 524288;   // 2^19 items
constexpr uint32_t kNoAllocMaxCells = 131072;  // 2^17 cells
constexpr size_t kNoAllocScratchBytes = sort_scratch_bytes(kNoAllocMaxItems, kNoAllocMaxCells);
static_assert(kNoAllocScratchBytes == 7340800, "scratch layout changed: update the documented size");

static __device__ __align__(256) unsigned char g_sort_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device: looked up afresh
// outside a capture (and cached), taken from the cache while `st` captures.
static pic_status scratch_address(cudaStream_t st, void** out) {
  int dev = 0;
  PIC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return (set_error("pic_sort_by_cell_noalloc: device %d out of range", dev), PIC_ERR_ARG);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  PIC_CUDA(cudaStreamIsCapturing(st, &cs));
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (cs != cudaStreamCaptureStatusNone) {
    if (!g_scratch_addr[dev])
      return (set_error("pic_sort_by_cell_noalloc: first call on device %d made during a stream capture; make one "
                        "call (n = 0 is enough) outside capture first", dev),
              PIC_ERR_STATE);
    *out = g_scratch_addr[dev];
    return PIC_OK;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "pic_sort_by_cell_noalloc: cudaGetSymbolAddress");
  if (!p) return (set_error("pic_sort_by_cell_noalloc: no device address for the scratch array"), PIC_ERR_CUDA);
  g_scratch_addr[dev] = p;
  *out = p;
  return PIC_OK;
}

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_sort_by_cell_noalloc(size_t n, const uint32_t* cell, const uint64_t* id, uint32_t n_cells,
                                               uint32_t* perm, uint32_t* cell_off, void* stream) {
  pic_status r = sort_by_cell_check(n, cell, id, n_cells, perm, cell_off, "pic_sort_by_cell_noalloc");
  if (r != PIC_OK) return r;
  if (n > kNoAllocMaxItems)
    return (set_error("pic_sort_by_cell_noalloc: %zu items exceed the limit of %zu", n, kNoAllocMaxItems), PIC_ERR_ARG);
  if (n_cells > kNoAllocMaxCells)
    return (set_error("pic_sort_by_cell_noalloc: %u cells exceed the limit of %u", n_cells, kNoAllocMaxCells),
            PIC_ERR_ARG);
  if (sort_scratch_bytes(n, n_cells) > kNoAllocScratchBytes)  // cannot happen within both limits (static_assert)
    return (set_error("pic_sort_by_cell_noalloc: scratch for %zu items and %u cells exceeds the limit of %zu bytes", n,
                      n_cells, kNoAllocScratchBytes),
            PIC_ERR_ARG);
  void* base = nullptr;
  r = scratch_address((cudaStream_t)stream, &base);
  if (r != PIC_OK) return r;
  // sort_by_cell_run clears the cell counts and status words it needs at
  // zero; every other scratch word it reads was written earlier in the call.
  return sort_by_cell_run(n, cell, id, n_cells, perm, cell_off, sort_scratch_layout(base, n, n_cells),
                          (cudaStream_t)stream);
}
