// Allocation-free entry point: Tr(K S), Tr(K D_x,y,z) of caller-owned device
// arrays, with the reduction scratch in a fixed device array of this library.
//
// Some callers cannot allocate device memory at the moment they need the
// traces: code that runs while a CUDA stream is being captured into a graph
// (allocation calls are not allowed there), or hosts whose framework owns all
// device memory and forbids a library from calling cudaMalloc behind its back.
// This entry point serves them: it takes only the caller's inputs and output
// and calls no cudaMalloc, cudaFree or allocating library routine.
//
// Scratch: one FP64 partial sum per (CTA, trace component) in g_trace_scratch,
// a file-scope device array of RT_NOALLOC_MAX_CTAS * 8 doubles (64 KiB) that
// every GPU loading the library holds until the process exits.  Each call
// writes every partial it later reads, so nothing has to start at zero; the
// array keeps the last call's partials.  All calls share the array: calls that
// overlap on the GPU (different streams, or different host threads on the same
// device) race on it and must be serialised by the caller.
#include <mutex>

#include "rt_internal.cuh"

namespace rt {

// the partial-sum pass of the trace reduction (elementwise.cu)
__global__ void k_traces(const double2* __restrict__ K, int64_t nnzb, const int32_t* __restrict__ rowidx,
                         const int32_t* __restrict__ col, const int32_t* __restrict__ bsize, int B,
                         const double* __restrict__ S, const int32_t* __restrict__ ks_map,
                         const double* __restrict__ Dx, const double* __restrict__ Dy, const double* __restrict__ Dz,
                         const int32_t* __restrict__ kd_map, double* __restrict__ part);

namespace {

constexpr int kMaxCtas = RT_NOALLOC_MAX_CTAS;
constexpr int kThreads = 256;  // the block size k_traces is written for
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_trace_scratch[kMaxCtas * 8];

// Adds the partials of the first pass in a fixed order and writes the eight
// values (Re/Im of the four traces) to the caller's output.
__global__ void k_traces_final_out(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double s[8][kThreads];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < nb; i += kThreads)
    for (int c = 0; c < 8; ++c) acc[c] += part[i * 8 + c];
  for (int c = 0; c < 8; ++c) s[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int off = kThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off)
      for (int c = 0; c < 8; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x < 8) out[threadIdx.x] = s[threadIdx.x][0];
}

std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_trace_scratch on the current device (looked up once per
// device; in host code the symbol itself is only a host-side stand-in).
rt_status scratch_for_current_device(double** out, const char** why) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();  // the error of this lookup itself (nothing was pending before it)
    *why = "no usable current CUDA device";
    return RT_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_trace_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();  // the error of this lookup itself (nothing was pending before it)
      *why = "cudaGetSymbolAddress of the scratch array failed";
      return RT_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return RT_OK;
}

// There is no context to hold a message: failures print their reason to stderr.
rt_status fail(rt_status code, const std::string& why) {
  fprintf(stderr, "rt_traces_noalloc: %s\n", why.c_str());
  return code;
}

}  // namespace
}  // namespace rt

extern "C" {

RT_API rt_status rt_traces_noalloc(const double* K, int64_t nnzb, const int32_t* rowidx, const int32_t* col,
                                   const int32_t* bsize, int32_t B, const double* S, const int32_t* ks_map,
                                   const double* Dx, const double* Dy, const double* Dz, const int32_t* kd_map,
                                   int32_t n_ctas, double* out, void* cuda_stream) {
  using namespace rt;
  if (!K || !rowidx || !col || !bsize || !S || !ks_map || !Dx || !Dy || !Dz || !kd_map || !out)
    return fail(RT_EINVAL, "NULL pointer argument");
  if (nnzb < 0 || B < 1 || B > 13) return fail(RT_EINVAL, "nnzb must be >= 0 and B in 1..13");
  int nb = n_ctas;
  if (nb == 0) {
    int64_t want = (nnzb + kThreads - 1) / kThreads;
    nb = (int)(want < 1 ? 1 : (want > kMaxCtas ? kMaxCtas : want));
  }
  if (nb < 1 || nb > kMaxCtas)
    return fail(RT_EINVAL, "n_ctas = " + std::to_string(n_ctas) + " is outside 1.." + std::to_string(kMaxCtas) +
                               " (the scratch holds RT_NOALLOC_MAX_CTAS partial sums)");
  // An error left pending by the caller's earlier work is reported as such and
  // left in place (not consumed): only errors of this call's own launches are
  // read and cleared below.
  cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess)
    return fail(RT_ECUDA, std::string("a CUDA error from earlier work is pending (not cleared): ") +
                              cudaGetErrorString(pending));
  double* scratch = nullptr;
  const char* why = nullptr;
  rt_status st = scratch_for_current_device(&scratch, &why);
  if (st != RT_OK) return fail(st, why);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  k_traces<<<nb, kThreads, 0, s>>>(reinterpret_cast<const double2*>(K), nnzb, rowidx, col, bsize, B, S, ks_map, Dx,
                                   Dy, Dz, kd_map, scratch);
  k_traces_final_out<<<1, kThreads, 0, s>>>(scratch, nb, out);
  cudaError_t e = cudaGetLastError();  // nothing was pending before the launches: this error is theirs
  if (e != cudaSuccess) return fail(RT_ECUDA, std::string("launch failed: ") + cudaGetErrorString(e));
  return RT_OK;
}

}  // extern "C"
