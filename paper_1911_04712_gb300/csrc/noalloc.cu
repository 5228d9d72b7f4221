// dpd_forces_noalloc: pair forces on a caller-provided state without any
// device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// forces: code running inside a host callback or a custom allocator, a
// framework that has handed every byte of device memory to its own pool,
// or a real-time loop that must not hit cudaMalloc's implicit device
// synchronisation.  This entry point serves them: all the scratch it needs
// (float4 copies of the state, the cell counts and starts, the reorder keys)
// lives in one file-scope static device array of fixed size, reserved when
// the library is loaded and held by every GPU that loads it until the
// process exits.  The caller passes only its inputs and its output.
//
// The array's name is a host-side stand-in in host code, not a device
// address; the device address is looked up with cudaGetSymbolAddress once
// per device, on that device's first call (so that first call should come
// before any stream capture).  Every call shares the one array and leaves
// its contents behind; the counts that must start at zero are cleared at the
// start of each call.  Calls whose work overlaps on the GPU (different
// streams, or different host threads) race on the array and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "dpd.h"
#include "engine.h"
#include "kernels.h"

namespace dpd {

namespace {

constexpr int kNaMaxParticles = DPD_NOALLOC_MAX_PARTICLES;
constexpr int kNaMaxCells = DPD_NOALLOC_MAX_CELLS;
constexpr int kNaMaxSlices = kNaMaxCells * kSlicesX;  // entries of the cell list
constexpr int kNaScanTiles = (kNaMaxSlices + 1 + kScanTile - 1) / kScanTile;
constexpr size_t kNaCellCap = (size_t)kNaScanTiles * kScanTile;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffPos = 0;
constexpr size_t kOffVel = kOffPos + align256(sizeof(float4) * kNaMaxParticles);
constexpr size_t kOffFrc = kOffVel + align256(sizeof(float4) * kNaMaxParticles);
constexpr size_t kOffPos2 = kOffFrc + align256(sizeof(float4) * kNaMaxParticles);
constexpr size_t kOffVel2 = kOffPos2 + align256(sizeof(float4) * kNaMaxParticles);
constexpr size_t kOffCellOf = kOffVel2 + align256(sizeof(float4) * kNaMaxParticles);
constexpr size_t kOffSlotIn = kOffCellOf + align256(sizeof(int) * kNaMaxParticles);
constexpr size_t kOffKey = kOffSlotIn + align256(sizeof(int) * kNaMaxParticles);
constexpr size_t kOffCount = kOffKey + align256(sizeof(int) * kNaMaxParticles);
constexpr size_t kOffStart = kOffCount + align256(sizeof(int) * kNaCellCap);
constexpr size_t kOffBsum = kOffStart + align256(sizeof(int) * kNaCellCap);
constexpr size_t kOffState = kOffBsum + align256(sizeof(int) * kNaScanTiles);
constexpr size_t kOffErr = kOffState + align256(sizeof(BoxState));
constexpr size_t kScratchBytes = kOffErr + align256(sizeof(unsigned));

}  // namespace

// The scratch: about 3.5 MB for 32768 particles and 32767 cells (two x slices each).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Zero the cell counts and the error word; set the step of the force.
__global__ void k_noalloc_reset(int ncell_padded, unsigned long long step) {
  int *count = reinterpret_cast<int *>(g_noalloc_scratch + kOffCount);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell_padded;
       c += gridDim.x * blockDim.x)
    count[c] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    BoxState *st = reinterpret_cast<BoxState *>(g_noalloc_scratch + kOffState);
    st->step = step;
    st->remaining = 0;
    st->pending = 0;
    st->adv = 1;
    *reinterpret_cast<unsigned *>(g_noalloc_scratch + kOffErr) = 0u;
  }
}

// Device address of the scratch on each device, looked up once per device
// and kept for the life of the process (a cudaDeviceReset, which may load
// the module again at another address, is not supported).
static unsigned char *scratch_address(int device, int *status) {
  static std::mutex mu;
  static unsigned char *addr[64] = {nullptr};
  std::lock_guard<std::mutex> g(mu);
  if (device < 0 || device >= 64) {
    *status = set_error(DPD_ERR_CUDA, "device ordinal %d out of range", device);
    return nullptr;
  }
  if (!addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      *status = set_error(DPD_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s",
                          cudaGetErrorString(e));
      return nullptr;
    }
    addr[device] = static_cast<unsigned char *>(p);
  }
  *status = DPD_OK;
  return addr[device];
}

}  // namespace dpd

extern "C" int dpd_forces_noalloc(int64_t n, const float *pos, const float *vel,
                                  const double box[3], double a, double gamma, double kT,
                                  double rc, double dt, uint64_t seed, uint64_t step,
                                  float *force, void *stream) {
  using namespace dpd;
  clear_error();
  if (!box) return set_error(DPD_ERR_ARG, "null box");
  if (n < 0) return set_error(DPD_ERR_ARG, "negative particle count");
  if (n > kNaMaxParticles)
    return set_error(DPD_ERR_ARG,
                     "dpd_forces_noalloc handles at most %d particles (got %lld); use the "
                     "allocating context API for larger systems",
                     kNaMaxParticles, (long long)n);
  BoxParams bp{};
  for (int k = 0; k < 3; ++k) bp.L[k] = box[k];
  bp.a = a;
  bp.gamma = gamma;
  bp.kT = kT;
  bp.rc = rc;
  bp.dt = dt;
  bp.mass = 1.0;
  bp.kexp = 1.0;
  bp.fb_flow = 2;
  bp.seed = seed;
  int nc[3];
  int rc_ = check_params(bp, nc);
  if (rc_) return rc_;
  const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];  // x slices of the cells
  if (ncell > kNaMaxSlices)
    return set_error(DPD_ERR_ARG,
                     "dpd_forces_noalloc handles at most %d cells (box has %lld); use the "
                     "allocating context API for larger boxes",
                     kNaMaxCells, (long long)(ncell / kSlicesX));
  if (n == 0) return DPD_OK;
  if (!pos || !vel || !force) return set_error(DPD_ERR_ARG, "null device pointer");

  int dev = -1;
  DPD_CUDA_TRY(cudaGetDevice(&dev));
  int status = DPD_OK;
  unsigned char *base = scratch_address(dev, &status);
  if (!base) return status;

  cudaStream_t s = (cudaStream_t)stream;
  Packed P{};
  P.pos = reinterpret_cast<float4 *>(base + kOffPos);
  P.vel = reinterpret_cast<float4 *>(base + kOffVel);
  P.frc = reinterpret_cast<float4 *>(base + kOffFrc);
  P.pos2 = reinterpret_cast<float4 *>(base + kOffPos2);
  P.vel2 = reinterpret_cast<float4 *>(base + kOffVel2);
  P.cellOf = reinterpret_cast<int *>(base + kOffCellOf);
  P.slotIn = reinterpret_cast<int *>(base + kOffSlotIn);
  P.keyTmp = reinterpret_cast<int *>(base + kOffKey);
  P.count = reinterpret_cast<int *>(base + kOffCount);
  P.start = reinterpret_cast<int *>(base + kOffStart);
  P.bsum = reinterpret_cast<int *>(base + kOffBsum);
  P.boxes = nullptr;
  P.pbase = nullptr;
  P.st = reinterpret_cast<BoxState *>(base + kOffState);
  P.err = reinterpret_cast<unsigned *>(base + kOffErr);
  P.ntot = (int)n;
  P.ncell = (int)ncell;
  P.nbox = 1;
  P.single = make_box_dev(bp, 0, 0, (int)n);

  const int padded = scan_tiles((int)ncell) * kScanTile;
  k_noalloc_reset<<<(padded + 255) / 256, 256, 0, s>>>(padded, (unsigned long long)step);
  DPD_CUDA_TRY(cudaGetLastError());
  DPD_CUDA_TRY(launch_load(P, 0, (int)n, pos, vel, P.single.L[0], P.single.L[1], P.single.L[2], s));
  StepConfig cfg{};
  DPD_CUDA_TRY(launch_step(P, false, false, cfg, s));
  DPD_CUDA_TRY(launch_gather(P, 0, 0, (int)n, nullptr, nullptr, force, s));
#if defined(DPD_CHECKED) && DPD_CHECKED
  // checked build: read the error word back (the normal build does not wait)
  unsigned h = 0;
  DPD_CUDA_TRY(cudaMemcpyAsync(&h, P.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  DPD_CUDA_TRY(cudaStreamSynchronize(s));
  if (h & kErrBounds)
    return set_error(DPD_ERR_INTERNAL, "a kernel's index check failed (checked build)");
#endif
  return DPD_OK;
}
