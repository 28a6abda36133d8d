// npfem_step_noalloc: the batched step for callers that cannot allocate device memory.
//
// Some callers of this library run where cudaMalloc is off limits: inside a host
// framework that owns every device allocation through its own pool, in code that runs
// while a stream is being captured, or in tools whose device memory budget is fixed at start-up.
// They can still hand us their state arrays.  This entry point needs no workspace from
// the caller and asks the CUDA runtime for none: the per-warp workspace, the work-queue
// counter and the per-cell layout live in one file-scope device array of fixed size,
// reserved when the library is loaded (every GPU that loads the library holds it until
// the process exits).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/npfem.h"
#include "api_internal.h"
#include "step_kernel.cuh"

using namespace npfem;

namespace {

// 32 MiB of static workspace per device.
constexpr size_t kStaticBytes = size_t(32) << 20;
constexpr int kStaticMaxCells = 65536;
constexpr size_t kCounterOff = 0;
constexpr size_t kPhaseOff = 64;  // per-phase cycle counters (telemetry, not read back here)
constexpr size_t kOffsetsOff = 256;
constexpr size_t kCellsOff = kOffsetsOff + sizeof(int64_t) * (kStaticMaxCells + 1);
constexpr size_t kSlotsOff = (kCellsOff + sizeof(int32_t) * kStaticMaxCells + 255) & ~size_t(255);
constexpr int kWarpsPerBlock = 4;
constexpr int kMaxDevices = 64;
constexpr size_t kSmemLimit = 72 * 1024;

static __device__ __align__(256) unsigned char g_npfem_static_scratch[kStaticBytes];

std::mutex g_setup_mutex;

// Cells 0..ncells-1, cell i owning vertices [i*n, (i+1)*n).
__global__ void fill_contiguous_layout(int64_t* offsets, int32_t* cells, int ncells, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= ncells; i += gridDim.x * blockDim.x) {
    offsets[i] = (int64_t)i * n;
    if (i < ncells) cells[i] = i;
  }
}

// On every call, with the call's device current: the device address of the static array
// (its host-side name is only a stand-in) and the shared-memory opt-in of the kernels.
// Neither allocates, and neither is cached, so a call after a device reset (a new primary
// context) finds the array and the kernel attribute of that context.
npfem_status setup_device(unsigned char** base, std::string* err) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_npfem_static_scratch);
  if (e != cudaSuccess) {
    *err = std::string("step_noalloc: cudaGetSymbolAddress of the static workspace failed: ") +
           cudaGetErrorString(e);
    return NPFEM_ERR_CUDA;
  }
  e = cudaFuncSetAttribute(npfem_step_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(npfem_step_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
  if (e != cudaSuccess) {
    *err = std::string("step_noalloc: cudaFuncSetAttribute failed: ") + cudaGetErrorString(e);
    return NPFEM_ERR_CUDA;
  }
  *base = static_cast<unsigned char*>(p);
  return NPFEM_OK;
}

}  // namespace

extern "C" npfem_status npfem_step_noalloc(const npfem_cell_type* type, npfem_precision prec, int32_t ncells,
                                           void* x, void* v, const void* f_ext, const int32_t* iters,
                                           const npfem_solver_opts* opts, double* residual_out,
                                           int32_t* status_out, void* stream) {
  std::string err;
  if (!type || !opts) return npfem_internal_fail(NPFEM_ERR_INVALID_ARG, "step_noalloc: null type or opts");
  if (prec != NPFEM_FP64 && prec != NPFEM_FP32FORM)
    return npfem_internal_fail(NPFEM_ERR_INVALID_ARG, "step_noalloc: bad precision");
  if (ncells < 0 || opts->iters < 0 || opts->alpha_log_len < 0 || (opts->alpha_log_len > 0 && !opts->alpha_log))
    return npfem_internal_fail(NPFEM_ERR_INVALID_ARG, "step_noalloc: negative size or bad alpha log");
  if (!(opts->tol >= 0.0) || std::isinf(opts->tol))
    return npfem_internal_fail(NPFEM_ERR_INVALID_ARG, "step_noalloc: tol must be finite and >= 0");
  if (ncells > kStaticMaxCells)
    return npfem_internal_fail(NPFEM_ERR_UNSUPPORTED,
                               "step_noalloc: " + std::to_string(ncells) + " cells exceed the static limit of " +
                                   std::to_string(kStaticMaxCells) + " cells per call");
  if (ncells == 0) return NPFEM_OK;
  if (!x || !v || !f_ext) return npfem_internal_fail(NPFEM_ERR_INVALID_ARG, "step_noalloc: null state array");
  const HostType& H = type->host;
  const size_t ssize = prec == NPFEM_FP64 ? sizeof(double) : sizeof(float);
  const size_t zbytes = sizeof(double) * 3 * ((size_t)H.n + 1);
  const int z_in_smem = zbytes * kWarpsPerBlock <= kSmemLimit ? 1 : 0;
  size_t slot = ssize * ((8 + 2 * (size_t)kHistory) * 3 * (size_t)H.n + 9 * (size_t)H.T + 3 * (size_t)H.E);
  slot = (slot + 255) & ~size_t(255);
  if (!z_in_smem) slot += zbytes;
  slot = (slot + 255) & ~size_t(255);
  const size_t avail = kStaticBytes - kSlotsOff;
  const size_t slots_fit = avail / slot;
  if (slots_fit < (size_t)kWarpsPerBlock)
    return npfem_internal_fail(NPFEM_ERR_UNSUPPORTED,
                               "step_noalloc: cell type needs " + std::to_string(slot) + " bytes of workspace per "
                               "warp; the static workspace holds " + std::to_string(avail) + " bytes (" +
                               std::to_string(kWarpsPerBlock) + " warps minimum)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return npfem_internal_fail(NPFEM_ERR_CUDA, "step_noalloc: no usable current device");
  unsigned char* base = nullptr;
  npfem_status rc = setup_device(&base, &err);
  if (rc != NPFEM_OK) return npfem_internal_fail(rc, err);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = (int)std::min<size_t>(slots_fit / kWarpsPerBlock, (size_t)sms * 3);
  blocks = std::min(blocks, (ncells + kWarpsPerBlock - 1) / kWarpsPerBlock);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* counter = reinterpret_cast<int*>(base + kCounterOff);
  int64_t* offsets = reinterpret_cast<int64_t*>(base + kOffsetsOff);
  int32_t* cells = reinterpret_cast<int32_t*>(base + kCellsOff);
  // the queue head must start at zero; the layout arrays are rewritten every call
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return npfem_internal_fail(NPFEM_ERR_CUDA, std::string("step_noalloc: ") + cudaGetErrorString(e));
  fill_contiguous_layout<<<(ncells + 256) / 256, 256, 0, st>>>(offsets, cells, ncells, H.n);
  StepParams P{};
  P.ncells_list = ncells;
  P.cell_list = cells;
  P.offsets = offsets;
  P.n_total = (int64_t)ncells * H.n;
  P.iters = iters;
  P.iters_default = opts->iters;
  P.residual_out = residual_out;
  P.status_out = status_out;
  P.tol = opts->tol;
  P.iters_done = opts->iters_done;
  P.alpha_log = opts->alpha_log;
  P.alpha_log_len = opts->alpha_log_len;
  P.queue_counter = counter;
  P.phase_cycles = reinterpret_cast<unsigned long long*>(base + kPhaseOff);
  P.scratch = reinterpret_cast<char*>(base + kSlotsOff);
  P.slot_bytes = slot;
  P.z_in_smem = z_in_smem;
  P.solve_per_coord = 0;
  P.solve_cells = 1;
  const size_t smem = z_in_smem ? zbytes * kWarpsPerBlock : 0;
  if (prec == NPFEM_FP64)
    npfem_step_kernel<double><<<blocks, 32 * kWarpsPerBlock, smem, st>>>(
        type->v64, P, static_cast<double*>(x), static_cast<double*>(v), static_cast<const double*>(f_ext));
  else
    npfem_step_kernel<float><<<blocks, 32 * kWarpsPerBlock, smem, st>>>(
        type->v32, P, static_cast<float*>(x), static_cast<float*>(v), static_cast<const float*>(f_ext));
  e = cudaGetLastError();
  if (e != cudaSuccess) return npfem_internal_fail(NPFEM_ERR_CUDA, std::string("step_noalloc: ") + cudaGetErrorString(e));
  return NPFEM_OK;
}
