// Allocation-free scoring entry point for small volumes.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or allocator hooks, real-time loops where an
// allocation may block or fail at the worst moment, or processes that sit
// under a strict device-memory budget.  cs_ngf_score_rotations_noalloc serves
// them.  It runs the same kernels as cs_ngf_score_rotations, one rotation at a
// time, but all of its scratch memory (the fixed-volume spectra, the resampled
// volume, the FFT intermediates, the twiddle tables and the per-rotation
// result key) lives in one file-scope device array of fixed size, g_scratch.
// Every GPU that loads this library holds that array until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/cs_ngf.h"
#include "kernels.cuh"

using namespace csngf;

namespace csngf {
void set_last_error(const std::string& msg);   // cs_ngf.cu
}

namespace {

constexpr int kNaMaxDim = CS_NGF_NOALLOC_MAX_DIM;   // per axis
constexpr int kNaMaxPad = 64;   // FFT length per axis (2 * 32 - 1 -> 64)

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// byte offsets inside the scratch array (every slice 256-byte aligned)
constexpr size_t kUVBytes = align256((size_t)7 * (kNaMaxPad / 2 + 1) * kNaMaxPad * kNaMaxPad * 8);
constexpr size_t kF02Elems = (size_t)4 * kNaMaxDim * kNaMaxDim * kNaMaxPad;               // >= (2n-1) P P
constexpr size_t kF13Elems = (size_t)4 * kNaMaxDim * kNaMaxPad * kNaMaxPad;               // >= (2n-1)^2 P
constexpr size_t kF02Bytes = align256(kF02Elems * 8);
constexpr size_t kF13Bytes = align256(kF13Elems * 8);
constexpr size_t kVolBytes = align256((size_t)kNaMaxDim * kNaMaxDim * kNaMaxDim * 4);
constexpr size_t kMaskBytes = align256((size_t)kNaMaxDim * kNaMaxDim * kNaMaxDim);
constexpr size_t kBQBytes = align256((size_t)kNaMaxDim * kNaMaxDim * kNaMaxDim * 16);
constexpr size_t kC8Bytes = align256((size_t)kNaMaxDim * kNaMaxDim * kNaMaxDim);
constexpr size_t kTwBytes = align256((size_t)3 * kNaMaxPad * 8);
constexpr size_t kMiscBytes = 256;   // msum[2] (A, B), thr, key, rotation matrix

constexpr size_t kOffUV = 0;
constexpr size_t kOffF02 = kOffUV + kUVBytes;
constexpr size_t kOffF13 = kOffF02 + kF02Bytes;
constexpr size_t kOffBh = kOffF13 + kF13Bytes;
constexpr size_t kOffMh = kOffBh + kVolBytes;
constexpr size_t kOffBQ = kOffMh + kMaskBytes;
constexpr size_t kOffC8 = kOffBQ + kBQBytes;
constexpr size_t kOffTw = kOffC8 + kC8Bytes;
constexpr size_t kOffMisc = kOffTw + kTwBytes;
constexpr size_t kScratchBytes = kOffMisc + kMiscBytes;
static_assert(kScratchBytes == (size_t)CS_NGF_NOALLOC_SCRATCH_BYTES, "header states the scratch size");

static_assert(kF02Elems >= (size_t)(2 * kNaMaxDim - 1) * kNaMaxPad * kNaMaxPad, "F2 fits");
static_assert(kF13Elems >= (size_t)(2 * kNaMaxDim - 1) * (2 * kNaMaxDim - 1) * kNaMaxPad, "F3 fits");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Misc {
  int msum[2];                 // [0] sum of M_A, [1] sum of the rotated M_B
  float thr;                   // overlap threshold in FFT units
  int pad_;
  unsigned long long key;      // best (score, shift) key of the current rotation
  RotMat rot;                  // the current rotation
};
static_assert(sizeof(Misc) <= kMiscBytes, "misc slice");

// device address of g_scratch per device ordinal, looked up once per device
constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[kMaxDevices] = {};

cs_ngf_status na_fail(cs_ngf_status s, const std::string& m) {
  set_last_error(m);      // reported by cs_ngf_last_error()
  return s;
}

#define NA_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return na_fail(CS_NGF_ECUDA, std::string(#call) + ": " +    \
                                                            cudaGetErrorString(e_));    \
  } while (0)

// FP64 twiddle tables exp(-2 pi i m / P) for the three axes, rounded to FP32
__global__ void k_na_twiddles(float2* tw, int Pz, int Py, int Px) {
  const int a = blockIdx.x, m = threadIdx.x;
  const int P = a == 0 ? Pz : (a == 1 ? Py : Px);
  if (m >= P) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)P, &s, &c);
  tw[a * kNaMaxPad + m] = make_float2((float)c, (float)(-s));
}

__global__ void k_na_set_rot(RotMat m, Misc* misc) {
  misc->rot = m;
  misc->msum[1] = 0;
  misc->key = 0ull;
}

__global__ void k_na_threshold(Misc* misc, float gamma, double pvol) {
  const int mn = min(misc->msum[0], misc->msum[1]);
  double t = ceil((double)gamma * (double)mn);
  if (t < 1.0) t = 1.0;
  misc->thr = (float)((t - 0.5) * pvol);
}

void quat_matrix(const double* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  const double s = std::sqrt(w * w + x * x + y * y + z * z);
  w = w / s;
  x = x / s;
  y = y / s;
  z = z / s;
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - w * z);
  R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);
  R[7] = 2.0 * (y * z + w * x);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
  const double targets[3] = {-1.0, 0.0, 1.0};
  for (double tgt : targets)
    for (int i = 0; i < 9; ++i)
      if (std::fabs(R[i] - tgt) <= 1e-9) R[i] = tgt;
}

int na_pad(int n) {
  const int pads[3] = {16, 32, 64};
  for (int p : pads)
    if (p >= 2 * n - 1) return p;
  return 0;
}

#define NA_DISPATCH(P, CALL)                       \
  switch (P) {                                     \
    case 16: { constexpr int PP = 16; CALL; } break; \
    case 32: { constexpr int PP = 32; CALL; } break; \
    case 64: { constexpr int PP = 64; CALL; } break; \
    default: break;                                \
  }

// a pointer the kernels will dereference must be device (or managed) memory
// of the device that runs them; anything else would fault instead of failing
cs_ngf_status na_check_ptr(const void* p, int device, const char* name) {
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return na_fail(CS_NGF_EINVAL, std::string(name) + ": cudaPointerGetAttributes: " +
                                      cudaGetErrorString(e));
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return na_fail(CS_NGF_EINVAL, std::string(name) + " is not device memory");
  if (at.device != device)
    return na_fail(CS_NGF_EINVAL, std::string(name) + " is on device " + std::to_string(at.device) +
                                      ", but device " + std::to_string(device) + " is current");
  return CS_NGF_OK;
}

cs_ngf_status na_launched(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(CS_NGF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return CS_NGF_OK;
}

}  // namespace

extern "C" cs_ngf_status cs_ngf_score_rotations_noalloc(
    const float* A, const uint8_t* maskA, const float* B, const uint8_t* maskB,
    const int32_t dims[3], float eps, float gamma, const double* quats, int32_t R,
    float* best_score, int32_t* best_shift, void* stream) {
  set_last_error("");
  if (!A || !maskA || !B || !maskB || !dims || !quats || !best_score || !best_shift)
    return na_fail(CS_NGF_EINVAL, "a pointer argument is NULL");
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 2 || dims[a] > kNaMaxDim)
      return na_fail(CS_NGF_EINVAL, "dims must be in [2, " + std::to_string(kNaMaxDim) +
                                        "] for the allocation-free entry point, got " +
                                        std::to_string(dims[a]));
  if (!(eps > 0.0f) || !std::isfinite(eps)) return na_fail(CS_NGF_EINVAL, "eps must be > 0");
  if (!(gamma > 0.0f && gamma <= 1.0f)) return na_fail(CS_NGF_EINVAL, "gamma must be in (0, 1]");
  if (R <= 0) return na_fail(CS_NGF_EINVAL, "R must be positive");
  for (int r = 0; r < R; ++r) {
    const double* q = quats + 4 * r;
    const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(std::fabs(n - 1.0) <= 1e-3))
      return na_fail(CS_NGF_EINVAL, "quaternion " + std::to_string(r) + " is not unit");
  }

  // set-up, once per device and with that device current: the device address
  // of g_scratch (the host-side symbol is only a stand-in for it)
  int device = 0;
  NA_CUDA(cudaGetDevice(&device));
  if (device < 0 || device >= kMaxDevices) return na_fail(CS_NGF_EINVAL, "device ordinal out of range");
  {
    const void* ptrs[6] = {A, maskA, B, maskB, best_score, best_shift};
    const char* names[6] = {"A", "maskA", "B", "maskB", "best_score", "best_shift"};
    for (int i = 0; i < 6; ++i)
      if (cs_ngf_status s = na_check_ptr(ptrs[i], device, names[i])) return s;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p)
        return na_fail(CS_NGF_ECUDA, std::string("cudaGetSymbolAddress(g_scratch): ") +
                                         cudaGetErrorString(e));
      g_na_ptr[device] = (unsigned char*)p;
    }
    base = g_na_ptr[device];
  }

  Geo g{};
  g.nz = dims[0]; g.ny = dims[1]; g.nx = dims[2];
  g.Pz = na_pad(g.nz); g.Py = na_pad(g.ny); g.Px = na_pad(g.nx);
  g.vz = 2 * g.nz - 1; g.vy = 2 * g.ny - 1; g.vx = 2 * g.nx - 1;
  g.eps2 = eps * eps;
  g.nvox = (long long)g.nz * g.ny * g.nx;
  g.nch = 3;                         // Eq. 2 (squared) measure
  g.nf = 4;
  g.store = kStoreF32;
  for (int j = 0; j < 4; ++j) g.scale0[j] = g.scale1[j] = 1.0f;

  float2* UV = (float2*)(base + kOffUV);
  float2* F02 = (float2*)(base + kOffF02);
  float2* F13 = (float2*)(base + kOffF13);
  float* Bh = (float*)(base + kOffBh);
  uint8_t* Mh = (uint8_t*)(base + kOffMh);
  float4* BQ = (float4*)(base + kOffBQ);
  uint8_t* C8 = (uint8_t*)(base + kOffC8);
  float2* tw = (float2*)(base + kOffTw);
  Misc* misc = (Misc*)(base + kOffMisc);
  cudaStream_t st = (cudaStream_t)stream;

  // fixed volume: twiddles, mask sum, forward transforms, weights (all in scratch)
  k_na_twiddles<<<3, kNaMaxPad, 0, st>>>(tw, g.Pz, g.Py, g.Px);
  if (cs_ngf_status s = na_launched("twiddles")) return s;
  const float2* twz = tw;
  const float2* twy = tw + kNaMaxPad;
  const float2* twx = tw + 2 * kNaMaxPad;
  NA_CUDA(cudaMemsetAsync(misc, 0, sizeof(Misc), st));
  k_copy_in<<<64, 256, 0, st>>>(A, maskA, g.nvox, Bh, Mh);
  if (cs_ngf_status s = na_launched("copy_in")) return s;
  k_mask_sum<<<64, 256, 0, st>>>(Mh, g.nvox, &misc->msum[0]);
  if (cs_ngf_status s = na_launched("mask_sum")) return s;
  NA_DISPATCH(g.Px, launch_fwd_x<PP>(Bh, Mh, F02, twx, g, 1, st));
  NA_DISPATCH(g.Py, launch_fwd_y<PP>(F02, F13, twy, g, 1, st));
  NA_DISPATCH(g.Pz, launch_prep_z<PP>(F13, UV, twz, g, st));
  if (cs_ngf_status s = na_launched("fixed transforms")) return s;

  k_pack_floating<<<64, 256, 0, st>>>(B, maskB, g, BQ, C8);
  if (cs_ngf_status s = na_launched("pack")) return s;
  const double pvol = (double)g.Px * (double)g.Py * (double)g.Pz;
  for (int r = 0; r < R; ++r) {
    double Rm[9];
    quat_matrix(quats + 4 * r, Rm);
    RotMat m;
    for (int i = 0; i < 9; ++i) m.m[i] = (float)Rm[i];
    k_na_set_rot<<<1, 1, 0, st>>>(m, misc);                 // also zeroes the sum and key
    k_resample<<<resample_grid(g, 1), 128, 0, st>>>(BQ, C8, &misc->rot, g, Bh, Mh, &misc->msum[1], nullptr);
    k_na_threshold<<<1, 1, 0, st>>>(misc, gamma, pvol);
    NA_DISPATCH(g.Px, launch_fwd_x<PP>(Bh, Mh, F02, twx, g, 1, st));
    NA_DISPATCH(g.Py, launch_fwd_y<PP>(F02, F13, twy, g, 1, st));
    NA_DISPATCH(g.Pz, launch_zmac<PP>(F13, UV, F02, twz, g, 1, nullptr, st));
    NA_DISPATCH(g.Py, launch_inv_y<PP>(F02, F13, twy, g, 1, nullptr, st));
    NA_DISPATCH(g.Px, launch_inv_x<PP>(F13, &misc->thr, &misc->key, nullptr, twx, g, 1, nullptr, st));
    k_finalize<<<1, 32, 0, st>>>(&misc->key, 1, g, best_score + r, best_shift + 3 * (size_t)r);
    if (cs_ngf_status s = na_launched("rotation")) return s;
  }
  return CS_NGF_OK;
}
