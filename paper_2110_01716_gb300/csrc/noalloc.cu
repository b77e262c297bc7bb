// noalloc.cu -- an inner product that allocates nothing.
//
// sem_dot keeps its reduction partials in memory the mesh allocated.  Some
// callers cannot have the library allocate device memory at all: hosts whose
// device-memory budget is fixed when they start, and loops that cannot pay
// for the implicit device synchronisation of cudaMalloc/cudaFree.  For them
// sem_dot_noalloc computes the same unique-node inner product with its
// scratch (one partial sum per CTA and a ticket counter) in the static device
// array below, which every GPU that loads the library holds until the process
// exits.  The caller passes the inputs and the device location of the result.
#include <mutex>
#include <new>

#include "common.cuh"

namespace sem {

// Scratch: kNoAllocSlots partial sums (one per CTA) followed by the ticket
// counter of the last-CTA-finishes reduction.  64 KiB per device.
constexpr int kNoAllocSlots = 8190;
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocPointsPerThread = 32;
constexpr int64_t kNoAllocPointsPerCta = (int64_t)kNoAllocThreads * kNoAllocPointsPerThread;
constexpr size_t kNoAllocScratchBytes = 65536;
static_assert(kNoAllocSlots * sizeof(double) + sizeof(unsigned int) <= kNoAllocScratchBytes,
              "scratch layout does not fit");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// One CTA per kNoAllocPointsPerCta local points; each CTA writes its partial
// into its own slot and the last CTA to finish adds the slots in CTA order.
__global__ void __launch_bounds__(kNoAllocThreads)
    dot_noalloc_kernel(Topo t, const double *__restrict__ u, const double *__restrict__ v,
                       double *__restrict__ result, unsigned char *__restrict__ scratch) {
  double *slots = reinterpret_cast<double *>(scratch);
  unsigned int *ticket = reinterpret_cast<unsigned int *>(scratch + kNoAllocSlots * sizeof(double));
  __shared__ double sh[kNoAllocThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kNoAllocPointsPerCta;
  double acc = 0.0;
  for (int q = 0; q < kNoAllocPointsPerThread; ++q) {
    const int64_t l = base + (int64_t)q * kNoAllocThreads + threadIdx.x;
    if (l < t.nl) {
      const PointInfo p = point_info((uint32_t)l, t);
      acc = fma(scale_pow2_down(u[l], p.log2_mult), v[l], acc);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) sh[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kNoAllocThreads / 32; ++q) s += sh[q];
    slots[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(&slots[b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __syncthreads();
  if (lane == 0) sh[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double total = 0.0;
    for (int q = 0; q < kNoAllocThreads / 32; ++q) total += sh[q];
    *result = total;
  }
}

// Device address of the scratch array, looked up once per device (with that
// device current) on the first call made on it.
static unsigned char *noalloc_scratch_address() {
  static std::mutex mu;
  static unsigned char *addr[64] = {};
  int dev = 0;
  SEM_CHECK_CUDA(cudaGetDevice(&dev));
  SEM_REQUIRE(dev >= 0 && dev < 64, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    SEM_CHECK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    addr[dev] = static_cast<unsigned char *>(p);
  }
  return addr[dev];
}

}  // namespace sem

extern "C" sem_status sem_dot_noalloc(const sem_mesh *mesh, const double *u, const double *v,
                                      double *result, void *stream) {
  try {
    SEM_REQUIRE(mesh && u && v && result, "null argument");
    const sem::Topo &t = mesh->fine.t;
    const int64_t ctas = (t.nl + sem::kNoAllocPointsPerCta - 1) / sem::kNoAllocPointsPerCta;
    SEM_REQUIRE(ctas <= sem::kNoAllocSlots,
                "sem_dot_noalloc handles at most %lld local points (mesh has %lld); use sem_dot",
                (long long)sem::kNoAllocSlots * sem::kNoAllocPointsPerCta, (long long)t.nl);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *scratch = sem::noalloc_scratch_address();
    // the ticket counter must start at zero; the partial slots are overwritten
    SEM_CHECK_CUDA(cudaMemsetAsync(scratch + sem::kNoAllocSlots * sizeof(double), 0,
                                   sizeof(unsigned int), st));
    sem::dot_noalloc_kernel<<<(unsigned int)(ctas < 1 ? 1 : ctas), sem::kNoAllocThreads, 0, st>>>(
        t, u, v, result, scratch);
    SEM_CHECK_CUDA(cudaGetLastError());
    return SEM_OK;
  } catch (const sem::Failure &f) {
    return f.status;
  } catch (const std::bad_alloc &) {
    sem::set_error_message("host allocation failed");
    return SEM_ENOMEM;
  } catch (...) {
    // e.g. std::system_error from the lock: no exception crosses the C ABI
    sem::set_error_message("unexpected internal error");
    return SEM_ECUDA;
  }
}
