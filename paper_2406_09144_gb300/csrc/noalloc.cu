// Allocation-free PSF convolution.
//
// fr_psf_apply keeps its half spectra in a per-stream workspace that the library allocates
// with cudaMalloc on first use, and it needs a plan, whose creation allocates too. Some callers
// cannot allow that: code embedded in a host application that owns the whole device-memory
// budget through its own pool (a real-time imaging pipeline with a fixed, pre-reserved
// footprint), or code running where a cudaMalloc would implicitly synchronise the device or is
// forbidden by the host framework. fr_psf_convolve_noalloc serves them: it takes the PSF image
// and the skies as inputs, writes the convolved skies, and keeps every intermediate (twiddle
// tables, the PSF transfer function, the half spectra) in one file-scope device array of fixed
// size that is part of the library image, so no call allocates anything.
//
// The array is 32 MiB. Every GPU that loads the library holds it until the process exits. It
// fits images with nx * ny <= 2^20 pixels (nx, ny powers of two in [16, 8192]).
#include <algorithm>
#include <mutex>
#include <vector>

#include "fr_internal.cuh"

namespace fr {
namespace {

constexpr size_t NOALLOC_BYTES = size_t(32) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct DeviceScratch {
  int device;
  unsigned char* ptr;
};
std::mutex g_noalloc_mu;
std::vector<DeviceScratch> g_noalloc_dev;

// Device address of the scratch array for the current device. In host code the array's name is
// only a host-side stand-in, so the address must come from cudaGetSymbolAddress, once per
// device, with that device current.
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  FR_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  for (const DeviceScratch& d : g_noalloc_dev)
    if (d.device == dev) {
      *out = d.ptr;
      return FR_OK;
    }
  void* p = nullptr;
  FR_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  g_noalloc_dev.push_back({dev, (unsigned char*)p});
  *out = (unsigned char*)p;
  return FR_OK;
}

__global__ void noalloc_twiddles(float2* tw, int L) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)m / (double)L, &s, &c);
    tw[m] = make_float2((float)c, (float)s);
  }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace fr

using namespace fr;

extern "C" int fr_psf_convolve_noalloc(const float* psf, const float* sky, int32_t nx, int32_t ny,
                                       int32_t batch, float* out, void* stream) {
  if (!psf || !sky || !out || batch < 1) {
    set_error("psf, sky and out must be non-null and batch >= 1");
    return FR_EINVAL;
  }
  if (nx < 16 || ny < 16 || nx > 8192 || ny > 8192 || (nx & (nx - 1)) || (ny & (ny - 1))) {
    // the padded transforms of 2nx and 2ny points must be lengths the FFT passes take
    set_error("nx, ny must be powers of two in [16, 8192] (got %d x %d)", nx, ny);
    return FR_EINVAL;
  }
  // scratch: twiddles (2ny, 2nx), transfer TT [ny+1][2nx] f32, then a region used first for the
  // PSF half spectra [ny+1][2nx] and afterwards for one image's H [nx][ny+2] and HT [ny+1][nx]
  const size_t q = (size_t)ny + 1;
  const size_t o_twr = 0;
  const size_t o_twc = align256(o_twr + (size_t)2 * ny * sizeof(float2));
  const size_t o_tt = align256(o_twc + (size_t)2 * nx * sizeof(float2));
  const size_t o_reg = align256(o_tt + q * 2 * nx * sizeof(float));
  const size_t h_bytes = (size_t)nx * (ny + 2) * sizeof(float2);
  const size_t reg_bytes =
      std::max(q * 2 * nx * sizeof(float2), align256(h_bytes) + q * nx * sizeof(float2));
  if ((size_t)nx * ny > (size_t(1) << 20) || o_reg + reg_bytes > NOALLOC_BYTES) {
    set_error("fr_psf_convolve_noalloc: %d x %d exceeds the fixed scratch (nx * ny <= 2^20, "
              "%zu bytes needed, %zu available)",
              nx, ny, o_reg + reg_bytes, NOALLOC_BYTES);
    return FR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  FR_TRY(noalloc_scratch(&base));
  float2* tw_rows = (float2*)(base + o_twr);
  float2* tw_cols = (float2*)(base + o_twc);
  float* tt = (float*)(base + o_tt);
  float2* reg = (float2*)(base + o_reg);
  noalloc_twiddles<<<16, 256, 0, s>>>(tw_rows, 2 * ny);
  FR_LAUNCHED();
  noalloc_twiddles<<<16, 256, 0, s>>>(tw_cols, 2 * nx);
  FR_LAUNCHED();
  // every scratch element read below is written earlier in the same call: nothing needs zeroing
  FR_TRY(build_transfer(nx, ny, 1, psf, 2 * nx, 2 * ny, reg, tt, tw_rows, tw_cols, s));
  float2* h = reg;
  float2* ht = (float2*)((unsigned char*)reg + align256(h_bytes));
  const size_t npix = (size_t)nx * ny;
  for (int b = 0; b < batch; ++b) {
    PsfArgs a;
    a.nx = nx;
    a.ny = ny;
    a.lx = 2 * nx;
    a.ly = 2 * ny;
    a.nimg = 1;
    a.nsky = 1;
    a.hp = ny + 2;
    a.transfer = tt;
    a.sky = sky + b * npix;
    a.out = out + b * npix;
    a.dirty = nullptr;
    a.value = nullptr;
    FR_TRY(psf_apply_passes(a, h, ht, tw_rows, tw_cols, s));
  }
  return FR_OK;
}
