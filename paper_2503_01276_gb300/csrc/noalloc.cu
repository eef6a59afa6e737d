// Single-level effective coefficients without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a result: a process
// whose device memory is already reserved by another framework's caching allocator, a
// deployment with a fixed memory budget decided at start-up, or a latency-sensitive path
// where cudaMalloc/cudaFree would synchronise the whole device. mch_direct_noalloc serves
// them: it runs the same kernels as mch_solve_level for one level without a hierarchy
// (constraint setup, the persistent constrained solve, the Gram of the effective
// coefficients) but keeps every intermediate array in one fixed buffer compiled into the
// library. The caller passes the media and the output; nothing is allocated.
//
// The buffer is a file-scope __device__ array of MCH_NOALLOC_SCRATCH_BYTES, so every GPU
// that loads the library holds it until the process exits. In host code the array's name
// is only a host-side stand-in for the symbol, never a device address: every call looks up
// the device address with cudaGetSymbolAddress while the caller's device is current (a
// table lookup once the module is loaded), so no address is cached across calls, threads or
// a cudaDeviceReset. With CUDA's lazy module loading (the default) the driver creates the
// array when this file's module is first used on a device, and loads each kernel's code at its
// first launch: so the first call on a device, and the first call with another grid size or
// precision (other kernel instantiations), may allocate. A caller makes one call with the
// sizes and precision it will use at start-up, before its device memory is handed to a
// caching allocator; later calls with them allocate nothing. Calls on a capturing stream are
// refused (every call synchronises its stream to read the convergence record).
// All calls share the buffer and it keeps the last call's contents: the parts that must
// start at zero are cleared on every call, and calls that overlap on the GPU (on different
// streams, or from different host threads) race on it.
#include <cuda_runtime.h>

#include "../../include/mch.h"
#include "common.cuh"
#include "kernels.h"

namespace mch {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MCH_NOALLOC_SCRATCH_BYTES];

int ilog2i(int v) {
  int r = 0;
  while ((1 << (r + 1)) <= v) ++r;
  return r;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Folds the per-unit and per-point records into {status bits, breakdown, max ratio}.
__global__ void k_noalloc_summary(int npts, int R, const int *pstat, const int *ustat,
                                  const double *ratio, int *flags, double *maxratio) {
  int f = 0, b = 0;
  double mr = 0.0;
  for (int i = threadIdx.x; i < npts; i += blockDim.x) f |= pstat[i];
  for (int u = threadIdx.x; u < npts * R; u += blockDim.x) {
    b |= ustat[u];
    const double r = ratio[u];
    mr = (r == r) ? fmax(mr, r) : 1e300;
  }
  atomicOr(&flags[0], f);
  atomicOr(&flags[1], b);
  // ratios are non-negative, so their bit patterns order like the values
  atomicMax(reinterpret_cast<unsigned long long *>(maxratio), (unsigned long long)__double_as_longlong(mr));
}

}  // namespace
}  // namespace mch

using namespace mch;

extern "C" mch_status mch_direct_noalloc(int n_cont, int n_elem, int periods, double rve_len,
                                         int precision, double rtol, int n_points,
                                         const double *kappa, const uint8_t *labels, double *E,
                                         void *cuda_stream) {
  // the buffer's device address on the current device (loads the module on first use)
  void *sym = nullptr;
  if (cudaGetSymbolAddress(&sym, g_noalloc_scratch) != cudaSuccess || !sym) {
    cudaGetLastError();
    return MCH_ERR_CUDA;
  }
  const int d = 2, N = n_cont, n = n_elem, P = periods;
  if (N < 1 || N > MCH_MAX_CONT || n_points < 1 || !(rve_len > 0) || !kappa || !labels || !E ||
      (precision != MCH_FP64 && precision != MCH_MIXED) || rtol < 0)
    return MCH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return MCH_ERR_CUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) return MCH_ERR_ARG;
  const bool fp64 = precision == MCH_FP64;
  if (!level2d_supported(n, P, fp64)) return MCH_ERR_UNSUPPORTED;
  const int R = N * (1 + d), nc = N * P * P;
  if (nc > MCH_MAX_NC) return MCH_ERR_UNSUPPORTED;
  const int nv = nv_of(n);
  const size_t np = (size_t)n_points;

  // carve the fixed buffer; reject batches that do not fit
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t o_minv = take(np * nv * sizeof(double));
  const size_t o_G = take(np * nc * R * sizeof(double));
  const size_t o_S64 = take(np * nc * nc * sizeof(double));
  const size_t o_S32 = take(np * nc * nc * sizeof(float));
  const size_t o_Sacc = take(np * nc * nc * sizeof(double));
  const size_t o_bacc = take(np * nc * 3 * sizeof(double));
  const size_t o_pstat = take(np * sizeof(int));
  const size_t o_drop = take(np * sizeof(int));
  const size_t o_x = take(np * R * nv * sizeof(double));
  const size_t o_yc = take(np * R * nv * sizeof(double));
  const size_t o_it = take(np * R * sizeof(int));
  const size_t o_sw = take(np * R * sizeof(int));
  const size_t o_ustat = take(np * R * sizeof(int));
  const size_t o_ratio = take(np * R * sizeof(double));
  const size_t o_sum = take(4 * sizeof(double));
  if (off > (size_t)MCH_NOALLOC_SCRATCH_BYTES) return MCH_ERR_OOM;

  unsigned char *base = static_cast<unsigned char *>(sym);
  auto D = [&](size_t o) { return reinterpret_cast<double *>(base + o); };
  auto I = [&](size_t o) { return reinterpret_cast<int *>(base + o); };

  // clear what must start at zero: the solution and the stencil output (their boundary and
  // padding entries are read but never written), the summary, and the output E (the Gram
  // adds into it)
  cudaError_t e = cudaMemsetAsync(base + o_x, 0, np * R * nv * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + o_yc, 0, np * R * nv * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + o_sum, 0, 4 * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(E, 0, np * R * R * sizeof(double), st);
  if (e != cudaSuccess) return MCH_ERR_CUDA;

  SetupArgs sa{n_points, n, P, N, R, nc, rve_len / n, rve_len, kappa, labels, D(o_G), D(o_S64),
               reinterpret_cast<float *>(base + o_S32), I(o_pstat), I(o_drop), D(o_minv), nv,
               D(o_Sacc), D(o_bacc)};
  if (launch_setup2d(sa, st) != cudaSuccess) return MCH_ERR_CUDA;
  const double tol = rtol > 0 ? rtol : 1e-8;
  const int max_iter = 4 * n + 50;
  if (fp64) {
    LevelArgs<double> la{n_points, R, n, P, N, nc, nv, ilog2i(n / P), ilog2i(P), kappa, labels,
                         D(o_S64), D(o_S64), D(o_minv), D(o_G), nullptr, D(o_x), I(o_it),
                         I(o_sw), D(o_ratio), I(o_ustat), 1e-4f, max_iter, tol, 6, nullptr};
    e = launch_level2d<double>(la, st);
  } else {
    LevelArgs<float> la{n_points, R, n, P, N, nc, nv, ilog2i(n / P), ilog2i(P), kappa, labels,
                        reinterpret_cast<float *>(base + o_S32), D(o_S64), D(o_minv), D(o_G),
                        nullptr, D(o_x), I(o_it), I(o_sw), D(o_ratio), I(o_ustat), 1e-4f,
                        max_iter, tol, 6, nullptr};
    e = launch_level2d<float>(la, st);
  }
  if (e != cudaSuccess) return MCH_ERR_CUDA;
  ApplyArgs aa{n_points, R, n, 1, nv, kappa, D(o_x), nullptr, 0.0, D(o_yc)};
  if (launch_apply2d(aa, st) != cudaSuccess) return MCH_ERR_CUDA;
  if (launch_gram(n_points, R, nv, D(o_x), D(o_yc), 1.0 / (rve_len * rve_len), E, st) !=
      cudaSuccess)
    return MCH_ERR_CUDA;
  k_noalloc_summary<<<1, 256, 0, st>>>(n_points, R, I(o_pstat), I(o_ustat), D(o_ratio),
                                       I(o_sum), D(o_sum) + 1);
  if (cudaGetLastError() != cudaSuccess) return MCH_ERR_CUDA;
  int flags[2] = {0, 0};
  double maxratio = 0.0;
  if (cudaMemcpyAsync(flags, base + o_sum, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(&maxratio, base + o_sum + sizeof(double), sizeof(double),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MCH_ERR_CUDA;
  if (flags[0]) return MCH_ERR_DEGENERATE;
  if (flags[1]) return MCH_ERR_BREAKDOWN;
  if (!(maxratio < tol)) return MCH_ERR_NOT_CONVERGED;
  return MCH_OK;
}
