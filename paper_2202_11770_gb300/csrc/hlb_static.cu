// hlb_static.cu — total-mass reduction that allocates nothing.
//
// Some callers cannot allocate device memory where they need this number:
// a host framework whose allocator owns every byte of device memory, or a
// time-critical loop where cudaMalloc's implicit synchronisation is not
// acceptable.  This entry point is the FP64 mass reduction of hlb_reduce
// (per-block partial sums, then one fixed-order final sum) with its partial
// sums kept in a file-scope device array instead of a workspace.  The caller
// still owns the input populations and the output.
#include <mutex>

#include "hlb_internal.h"

using namespace hlb;

namespace {

constexpr int BLOCK = 256;
constexpr int64_t MAX_PARTIALS = HLB_STATIC_MAX_SITES / BLOCK;

// Partial sums of the blocks of the last call.  Every GPU that loads the
// library holds this 2 MiB array until the process exits.  Calls share it.
static __device__ __align__(256) double g_partials[MAX_PARTIALS];

// Device address of g_partials per device ordinal, looked up once with that
// device current (in host code the symbol itself is only a host stand-in).
// It belongs to the device's primary context: after a cudaDeviceReset it is
// stale, which the header states as a condition of use.
constexpr int MAX_DEVICES = 64;
void* g_addr[MAX_DEVICES] = {};
std::mutex g_mutex;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
  __syncthreads();
  return r;
}

// One partial per 256-site block: sum over its sites of sum_i h_i.
template <typename S>
__global__ void __launch_bounds__(BLOCK) k_mass_static(const S* __restrict__ f, int64_t n,
                                                       double* __restrict__ part) {
  __shared__ double sh[BLOCK / 32];
  const int64_t x = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  double d = 0;
  if (x < n) {
#pragma unroll
    for (int i = 0; i < Q; ++i) d += (double)to_real(f[(int64_t)i * n + x]);
  }
  const double s = block_sum(d, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out = n + sum of the nb partials, in a fixed order.
__global__ void __launch_bounds__(1024) k_mass_static_finish(const double* __restrict__ part, int64_t nb, int64_t n,
                                                             double* __restrict__ out) {
  __shared__ double sh[32];
  double v = 0;
  for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    *out = (double)n + r;
  }
}

int partials_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hlb_cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return hlb_fail(HLB_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess) return hlb_cuda_fail(e, "cudaGetSymbolAddress(g_partials)");
    g_addr[dev] = p;
  }
  *out = (double*)g_addr[dev];
  return HLB_OK;
}

template <typename S>
cudaError_t launch(const void* f, int64_t n, double* part, double* out, cudaStream_t st) {
  const int64_t nb = (n + BLOCK - 1) / BLOCK;
  k_mass_static<S><<<(unsigned)nb, BLOCK, 0, st>>>((const S*)f, n, part);
  k_mass_static_finish<<<1, 1024, 0, st>>>(part, nb, n, out);
  return cudaGetLastError();
}

}  // namespace

extern "C" int hlb_mass_static(const void* f, int32_t precision, int64_t n_sites, double* mass, hlb_stream stream) {
  if (!f || !mass) return hlb_fail(HLB_ERR_ARG, "null population or output pointer");
  if (n_sites < 1) return hlb_fail(HLB_ERR_ARG, "n_sites must be >= 1");
  if (n_sites > HLB_STATIC_MAX_SITES)
    return hlb_fail(HLB_ERR_ARG, "n_sites exceeds the static scratch limit of " +
                                     std::to_string((long long)HLB_STATIC_MAX_SITES) + " sites");
  double* part = nullptr;
  int rc = partials_address(&part);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (precision) {
    case HLB_FP32: e = launch<float>(f, n_sites, part, mass, st); break;
    case HLB_BF16: e = launch<__nv_bfloat16>(f, n_sites, part, mass, st); break;
    case HLB_FP16: e = launch<__half>(f, n_sites, part, mass, st); break;
    case HLB_FP64: e = launch<double>(f, n_sites, part, mass, st); break;
    default: return hlb_fail(HLB_ERR_ARG, "unknown precision");
  }
  if (e != cudaSuccess) return hlb_cuda_fail(e, "hlb_mass_static launch");
  return HLB_OK;
}
