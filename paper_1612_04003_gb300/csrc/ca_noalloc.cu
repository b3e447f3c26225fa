// ca_noalloc.cu -- ca_gram_project_noalloc: the Gram + projection pass
// (steps a2+a3) for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need this pass:
// code that runs while another component owns every device allocation (a
// host framework with its own memory pool, where a raw cudaMalloc would
// fragment or bypass that pool), code on a latency-critical path where an
// allocation's implicit device synchronisation is not acceptable, or code
// that is only allowed to enqueue work on a stream it was handed.  This entry
// point takes no context and never allocates: its scratch lives in one
// file-scope device array of fixed size, so every GPU that loads the library
// holds that array (CA_NOALLOC_SCRATCH_BYTES) until the process exits.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress and caches it; make that
// first call before any stream capture.  All calls share the array and it
// keeps the last call's contents: calls that overlap on the GPU (on different
// streams, or from different host threads without ordering) race on it.
#include <algorithm>
#include <mutex>

#include "ca_bcd.h"
#include "ca_kernels.cuh"

namespace {

constexpr int kMaxSb = 128;            // rows of Y
constexpr long long kMaxK = 262144;    // length of the contraction (columns of A)
constexpr int kSplits = 32;            // split-K partial count
constexpr int kMaxDevices = 64;

// Layout of the scratch array (byte offsets, each 256-aligned).
constexpr size_t kErrOff = 0;                                              // error word
constexpr size_t kV2Off = 256;                                             // kMaxK float2
constexpr size_t kPartOff = kV2Off + (size_t)kMaxK * 8;                    // kSplits x 128 x 128 doubles
constexpr size_t kPPartOff = kPartOff + (size_t)kSplits * 128 * 128 * 8;   // kSplits x 128 doubles
constexpr size_t kROff = kPPartOff + (size_t)kSplits * 128 * 8;            // 128 x 128 doubles
constexpr size_t kTotal = kROff + (size_t)128 * 128 * 8;

}  // namespace

#define CA_NOALLOC_SCRATCH_BYTES (((size_t)(6u << 20)) + (size_t)(512u << 10))
static_assert(kTotal <= CA_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[CA_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_setup_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return CA_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return CA_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return CA_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int ca_gram_project_noalloc(void* cuda_stream, int xfmt, int prec, const void* A,
                                       long long N, long long K, long long ld, const int* idx,
                                       int sb, const double* v, double* G, double* p) {
  if (!A || !idx || !v || !G || !p || N < 1 || K < 1 || ld < K || sb < 1) return CA_ERR_ARG;
  if (sb > kMaxSb || K > kMaxK) return CA_ERR_UNSUPPORTED;  // beyond the fixed scratch
  if (xfmt != CA_DENSE_F64 && xfmt != CA_DENSE_F32) return CA_ERR_ARG;
  if (prec == CA_GRAM_FP16_SCALED) return CA_ERR_UNSUPPORTED;  // per-row scales: no fixed room
  if (prec < CA_GRAM_F64 || prec > CA_GRAM_BF16X3) return CA_ERR_ARG;
  const bool tc = (xfmt == CA_DENSE_F32) &&
                  (prec == CA_GRAM_TF32 || prec == CA_GRAM_FP32_EXACT || prec == CA_GRAM_BF16X3);
  if (tc && ((ld & 3) != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0)) return CA_ERR_ARG;
  for (const void* q : {A, (const void*)idx, (const void*)v, (const void*)G, (const void*)p})
    if (!on_device(q)) return CA_ERR_ARG;
  unsigned char* base = nullptr;
  const int st0 = scratch_for_current_device(&base);
  if (st0 != CA_OK) return st0;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  unsigned* err = reinterpret_cast<unsigned*>(base + kErrOff);
  float2* v2 = reinterpret_cast<float2*>(base + kV2Off);
  void* part = base + kPartOff;
  double* ppart = reinterpret_cast<double*>(base + kPPartOff);
  double* R = reinterpret_cast<double*>(base + kROff);

  // only the error word must start at zero; every other region read below is
  // first written by this call
  if (cudaMemsetAsync(err, 0, sizeof(unsigned), stream) != cudaSuccess) return CA_ERR_CUDA;
  const long long natoms = (K + 31) / 32;
  int P, sbp;
  if (tc) {
    // tile height: the smallest of 32, 64, 128 rows that holds sb
    sbp = sb <= 32 ? 32 : (sb <= 64 ? 64 : 128);
    P = (int)std::min<long long>(kSplits, natoms);
    const long long Kp = natoms * 32;
    k_split<<<(unsigned)((Kp + 255) / 256), 256, 0, stream>>>(v, K, Kp, v2);
    // (k_split writes v2: the Gram launch waits for it before its first load)
    if (launch_gram_tc(static_cast<const float*>(A), ld, N, K, idx, sb, v2, P, sbp,
                       static_cast<float*>(part), ppart, err, prec == CA_GRAM_FP32_EXACT ? 1 : (prec == CA_GRAM_BF16X3 ? 2 : 0),
                       stream) != 0)
      return CA_ERR_CUDA;
  } else {
    sbp = (sb + 63) / 64 * 64;
    const int t = sbp / 64;
    const int ntiles = t * (t + 1) / 2;
    const long long cps = (natoms + kSplits - 1) / kSplits;
    P = (int)((natoms + cps - 1) / cps);
    launch_gram_simt(xfmt == CA_DENSE_F64, dim3(P, ntiles), stream, A, ld, N, K, idx, sb, v, cps,
                     sbp, static_cast<double*>(part), ppart, err);
  }
  SolveArgs sa{idx, N, 1, 0, sb, sbp, 0.0, 0.0, 0.0, 0.0, nullptr, nullptr, nullptr};
  const long long entries = (long long)sb * (sb + 1) / 2 + sb;
  launch_reduce(tc, (int)std::min<long long>((entries + 31) / 32, 256), 0, stream, part, ppart, P,
                sbp, R, nullptr, p, nullptr, 0, sa, err);
  k_symmetrize<<<(unsigned)(((long long)sb * sb + 255) / 256), 256, 0, stream>>>(R, sbp, sb, G);
  if (cudaGetLastError() != cudaSuccess) return CA_ERR_CUDA;
  unsigned host_err = 0;
  if (cudaMemcpyAsync(&host_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return CA_ERR_CUDA;
  if (host_err & CA_DEV_ERR_TIMEOUT) return CA_ERR_TIMEOUT;
  if (host_err & CA_DEV_ERR_ARG) return CA_ERR_ARG;
  return CA_OK;
}
