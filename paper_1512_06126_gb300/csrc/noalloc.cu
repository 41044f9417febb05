// Allocation-free variant of the c64 matrix-vector product.
//
// Some callers cannot allocate device memory at all: code running under an
// allocator-free policy (for example inside a host-side memory budget that forbids
// cudaMalloc after start-up, or a plug-in that may only use buffers handed to it).
// ie_matvec_noalloc serves them: it takes every operand as a device pointer and
// keeps its two FFT work arrays in one fixed, file-scope device array instead of
// cudaMalloc'd memory.  The array is sized kScratchBytes (64 MiB); every GPU that
// loads the library reserves it until the process exits.
#include "../../include/ie.h"

#include <mutex>
#include <utility>
#include <vector>

#include "contract.cuh"
#include "fft.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;

// Device-side work space shared by every call of ie_matvec_noalloc.  In host code
// this name is only a stand-in: host code must use the address returned by
// cudaGetSymbolAddress (scratch_address below), never the symbol itself.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
std::vector<std::pair<int, void *>> g_addr;  // (device, device address of g_scratch)

// Device address of the scratch array on the current device, looked up once per
// device (the lookup is not an allocation).
ie_status scratch_address(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return IE_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto &e : g_addr)
    if (e.first == dev) {
      *out = e.second;
      return IE_OK;
    }
  void *p = nullptr;
  const cudaError_t err = cudaGetSymbolAddress(&p, g_scratch);
  if (err != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return IE_ERR_CUDA;
  }
  g_addr.emplace_back(dev, p);
  *out = p;
  return IE_OK;
}

}  // namespace

extern "C" ie_status ie_matvec_noalloc(int nx, int ny, int nz, int nrhs, const void *qf_dev,
                                       const void *in_scale_dev, const void *out_scale_dev, const void *diag_dev,
                                       const void *x_dev, void *y_dev, void *stream) {
  if (nx < 1 || ny < 1 || nz < 1 || nrhs < 1 || nrhs > 4 || !qf_dev || !in_scale_dev || !out_scale_dev ||
      !x_dev || !y_dev || x_dev == y_dev)
    return IE_ERR_ARG;
  // shapes the contraction cannot stage are argument errors, found before any launch
  if (!ie::contract_fits(nz, nrhs, true)) return IE_ERR_ARG;
  const long long cz = (long long)nrhs * 3 * nz;
  const long long t1_elems = (long long)ny * 2 * nx * cz;
  const long long spec_elems = 4LL * nx * ny * cz;
  const long long need = (t1_elems + spec_elems) * (long long)sizeof(float2);
  if (need > (long long)kScratchBytes) return IE_ERR_SCRATCH;
  ie::FftPlan px, py;
  try {
    px = ie::make_plan(2 * nx);
    py = ie::make_plan(2 * ny);
  } catch (...) {
    return IE_ERR_ARG;
  }
  void *base = nullptr;
  const ie_status st = scratch_address(&base);
  if (st != IE_OK) return st;
  float2 *t1 = static_cast<float2 *>(base);
  float2 *spec = t1 + t1_elems;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float2 *x = static_cast<const float2 *>(x_dev);
  float2 *y = static_cast<float2 *>(y_dev);
  // Every element of t1 and spec that a later kernel reads is written earlier in the
  // same call, so nothing left over from a previous call is ever read.
  ie::launch_fft_rows_fwd<float>(x, static_cast<const float2 *>(in_scale_dev), t1, (int)cz, nz, ny, nx, px, s);
  ie::launch_fft_axis<float, false>(t1, spec, 1, ny, 2 * ny, 2LL * nx * cz, py, 1.0f, s);
  // a wait that runs out inside the contraction is recorded in the library's own error
  // word, which ie_noalloc_sync reports
  if (ie::launch_contract<float>(spec, static_cast<const float2 *>(qf_dev), nx, ny, nz, nrhs, (int)cz,
                                ie::kContractAuto, nullptr, s) != 0)
    return IE_ERR_CUDA;
  ie::launch_fft_axis<float, true>(spec, t1, 1, 2 * ny, ny, 2LL * nx * cz, py, 1.0f, s);
  ie::launch_fft_rows_inv<float>(t1, x, static_cast<const float2 *>(diag_dev),
                                 static_cast<const float2 *>(out_scale_dev), y, (int)cz, nz, ny, nx, px, s);
  return cudaGetLastError() == cudaSuccess ? IE_OK : IE_ERR_CUDA;
}

extern "C" ie_status ie_noalloc_sync(void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return IE_ERR_CUDA;
  const int e = ie::contract_take_error(nullptr, s);
  if (e < 0) return IE_ERR_CUDA;
  return e ? IE_ERR_TIMEOUT : IE_OK;
}
