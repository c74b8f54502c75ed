// asci_sort_accumulate_noalloc: sort-and-accumulate without any allocation.
//
// Some callers cannot allocate device memory while they call this library:
// processes whose device memory is already reserved by another allocator or
// held under a cap, and embedders (latency-bound or certified code paths) whose
// policy forbids allocating behind their back.  For them this entry point runs
// the same sort-and-accumulate as asci_sort_accumulate with every scratch
// buffer carved from one fixed device array that the library owns.
//
// The array below is a file-scope __device__ variable: every GPU that loads
// the library's device code holds it (kNoAllocBytes) until the process exits.
// Host code cannot use the name g_noalloc_scratch as a device address; every
// call looks the address up with cudaGetSymbolAddress, with the call's device
// current.  The lookup is a host-side query of the loaded module, and doing it
// on every call keeps the address right for whatever context is current (a
// primary context re-created after cudaDeviceReset holds a new copy of the
// array at a new address).  With CUDA's lazy module loading the module, and
// with it the array, is loaded on a device at the first lookup or launch: the
// first call on a device is where the array is committed.
#include <cuda_runtime.h>

#include <cstring>

#include "asci_internal.cuh"

namespace asci {
namespace {

constexpr size_t kNoAllocMaxPairs = ASCI_NOALLOC_MAX_PAIRS;
// Per pair: keys (3 x 8 B), values (2 x 8 B), sums (8 B), unpacked keys (16 B),
// staged inputs (24 B), run flags and positions (12 B); plus radix histograms,
// scan partials, the error word and alignment slack.
constexpr size_t kNoAllocBytes = kNoAllocMaxPairs * 104 + (2u << 20);

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array in the current context.
int noalloc_region(void **out) {
  void *ptr = nullptr;
  ASCI_TRY_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
  *out = ptr;
  return ASCI_OK;
}

bool device_accessible(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Packs (alpha, beta) into the 64-bit key; a word with a bit at or above 32
// does not fit and sets *bad.
__global__ void k_na_pack(const asci_det *d, size_t n, uint64_t *keys, unsigned *bad) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const asci_det x = d[i];
    if ((x.alpha | x.beta) >> 32) *bad = 1u;
    keys[i] = pack_key((uint32_t)x.alpha, (uint32_t)x.beta);
  }
}

__global__ void k_na_unpack(const uint64_t *keys, size_t n, asci_det *out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    asci_det d;
    d.alpha = key_alpha(keys[i]);
    d.beta = key_beta(keys[i]);
    out[i] = d;
  }
}

unsigned na_grid(size_t n) {
  size_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

// Work queued on `s` reads and writes the shared array; every return path
// waits for it, so that no call leaves work on the array behind it.
struct SyncOnExit {
  cudaStream_t s;
  ~SyncOnExit() { cudaStreamSynchronize(s); }
};

int sort_accumulate_noalloc(const asci_det *keys, const double *values, size_t n,
                            asci_det *out_keys, double *out_sums, size_t *out_n, cudaStream_t s) {
  void *region = nullptr;
  ASCI_TRY(noalloc_region(&region));
  SyncOnExit guard{s};
  Arena arena(s, region, kNoAllocBytes);  // bump mode: allocates nothing
  unsigned *bad;
  ASCI_TRY(arena.alloc(&bad, 1));
  ASCI_TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned), s));
  const asci_det *dk = keys;
  const double *dv = values;
  if (!device_accessible(keys)) {
    asci_det *t;
    ASCI_TRY(arena.alloc(&t, n));
    ASCI_TRY_CUDA(cudaMemcpyAsync(t, keys, n * sizeof(asci_det), cudaMemcpyDefault, s));
    dk = t;
  }
  if (!device_accessible(values)) {
    double *t;
    ASCI_TRY(arena.alloc(&t, n));
    ASCI_TRY_CUDA(cudaMemcpyAsync(t, values, n * sizeof(double), cudaMemcpyDefault, s));
    dv = t;
  }
  uint64_t *k0, *k1, *uk;
  double *v0, *v1, *us;
  asci_det *dok;
  ASCI_TRY(arena.alloc(&k0, n));
  ASCI_TRY(arena.alloc(&k1, n));
  ASCI_TRY(arena.alloc(&uk, n));
  ASCI_TRY(arena.alloc(&v0, n));
  ASCI_TRY(arena.alloc(&v1, n));
  ASCI_TRY(arena.alloc(&us, n));
  ASCI_TRY(arena.alloc(&dok, n));
  k_na_pack<<<na_grid(n), 256, 0, s>>>(dk, n, k0, bad);
  ASCI_CHECK_LAUNCH();
  unsigned hbad = 0;
  ASCI_TRY_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  if (hbad) {
    record_error("asci_sort_accumulate_noalloc: a key word has bits at or above 32", __FILE__,
                 __LINE__);
    return ASCI_EINVAL;
  }
  ASCI_TRY_CUDA(cudaMemcpyAsync(v0, dv, n * sizeof(double), cudaMemcpyDefault, s));
  size_t u = 0;
  ASCI_TRY(sort_accumulate(&k0, &k1, &v0, &v1, n, uk, us, &u, arena));
  k_na_unpack<<<na_grid(u), 256, 0, s>>>(uk, u, dok);
  ASCI_CHECK_LAUNCH();
  ASCI_TRY_CUDA(cudaMemcpyAsync(out_sums, us, u * sizeof(double), cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaMemcpyAsync(out_keys, dok, u * sizeof(asci_det), cudaMemcpyDefault, s));
  ASCI_TRY_CUDA(cudaStreamSynchronize(s));
  *out_n = u;
  return ASCI_OK;
}

}  // namespace
}  // namespace asci

extern "C" int asci_sort_accumulate_noalloc(const asci_det *keys, const double *values, size_t n,
                                            asci_det *out_keys, double *out_sums, size_t *out_n,
                                            void *cuda_stream) {
  if (out_n) *out_n = 0;
  if (!keys || !values || !out_keys || !out_sums || !out_n) return ASCI_EINVAL;
  if (n > ASCI_NOALLOC_MAX_PAIRS) {
    asci::record_error("asci_sort_accumulate_noalloc: more pairs than ASCI_NOALLOC_MAX_PAIRS",
                       __FILE__, __LINE__);
    return ASCI_EINVAL;
  }
  if (n == 0) return ASCI_OK;
  return asci::sort_accumulate_noalloc(keys, values, n, out_keys, out_sums, out_n,
                                       (cudaStream_t)cuda_stream);
}
