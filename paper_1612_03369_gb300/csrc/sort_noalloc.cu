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
// The array is a file-scope __device__ variable, so every GPU that loads
// the library holds it (kNoAllocScratchBytes, 7 MiB) until the process exits.
// Host code must not use the array's name as a device address: it is a
// host-side stand-in.  The device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device; make that first call outside any stream
// capture.  All calls share the one array and it keeps the last call's
// contents, so calls whose work overlaps on the GPU (different streams, or
// host threads without ordering between them) race: order them.
#include <mutex>

#include "pic_internal.cuh"

namespace pic {

// Limits of the no-allocation sort.  The scratch for n items and C cells is
// about 12 B per item plus 8 B per cell (sort_scratch_bytes); at the limits
// below it fits in the 7 MiB array.
constexpr size_t kNoAllocMaxItems = 524288;   // 2^19 items
constexpr uint32_t kNoAllocMaxCells = 131072;  // 2^17 cells
constexpr size_t kNoAllocScratchBytes = size_t(7) << 20;

static __device__ __align__(256) unsigned char g_sort_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device (set-up on first use).
static pic_status scratch_address(void** out) {
  int dev = 0;
  PIC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return (set_error("pic_sort_by_cell_noalloc: device %d out of range", dev), PIC_ERR_ARG);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "pic_sort_by_cell_noalloc: cudaGetSymbolAddress");
    if (!p) return (set_error("pic_sort_by_cell_noalloc: no device address for the scratch array"), PIC_ERR_CUDA);
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
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
  if (sort_scratch_bytes(n, n_cells) > kNoAllocScratchBytes)
    return (set_error("pic_sort_by_cell_noalloc: scratch for %zu items and %u cells exceeds %zu bytes", n, n_cells,
                      kNoAllocScratchBytes),
            PIC_ERR_ARG);
  void* base = nullptr;
  r = scratch_address(&base);
  if (r != PIC_OK) return r;
  // sort_by_cell_run clears the cell counts and status words it needs at
  // zero; every other scratch word it reads was written earlier in the call.
  return sort_by_cell_run(n, cell, id, n_cells, perm, cell_off, sort_scratch_layout(base, n, n_cells),
                          (cudaStream_t)stream);
}
