// Kernels of the all-shift NGF correlation hot path (Cross-Sim-NGF,
// Sections 3.1-3.2).  Per rotation of the floating volume B:
//
//   resample   B_hat = B o T_theta (trilinear) and the rotated mask    (Sec. 3.2)
//   fwd_x      NGF of B_hat (Eq. 1), the six Eq. 6 channels and the mask,
//              packed as four complex fields, x-axis FFT
//   fwd_y      y-axis FFT
//   zmac       z-axis FFT, the spectral multiply-accumulate against the
//              fixed volume's spectra (Eq. 7-8, summed before the inverse),
//              z-axis inverse FFT of X + iY (numerator and overlap count)
//   inv_y      y-axis inverse FFT
//   inv_x      x-axis inverse FFT, s = X / N over the valid shifts (Eq. 5,
//              minimum overlap gamma), per-rotation argmax
//
// Data layout (all [slow]...[fast], complex64 = float2):
//   Bh, Mh   [r][z][y][x]                     float / uint8
//   F0       [r][j][z][y][kx]     j < nf       x transformed
//   F1       [r][j][kx][z][ky]                  x, y transformed
//   F2       [r][kx][vz][ky]                    Z = X + iY after the z inverse
//   F3       [r][vz][vy][kx]                    after the y inverse
//   UV       [2nch+1][kx <= Px/2][ky][kz]      fixed-volume weights (prepare)
// vz, vy, vx index the shift chi = v - (n - 1) in [-(n-1), n-1].
//
// Packed channel pairs (Eq. 2, squared measure): j=0 (xx, yy), j=1 (zz, xy),
// j=2 (xz, yz), j=3 (mask, 0).  Eq. 3 (unsquared measure): j=0 (x, y),
// j=1 (z, 0), j=2 (mask, 0).  F0/F1 hold g.nf fields per rotation.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fft_core.cuh"

namespace csngf {

struct Geo {
  int nz, ny, nx;       // volume dims
  int Pz, Py, Px;       // FFT lengths per axis
  int vz, vy, vx;       // 2n - 1 shift extents
  float eps2;           // eps^2 (Eq. 1)
  long long nvox;       // nz*ny*nx
  int nch;              // packed channel fields: 3 (Eq. 2, squared) or 2 (Eq. 3, unsquared)
  int nf;               // fields per rotation: nch + 1 (the mask field is last)
  int store;            // channel fields of F0 / F1: kStoreF32, kStoreBF16 or kStoreF16
  // FP16 form: channel field j of F0 (F1) is stored as its value times
  // scale0[j] (scale1[j]), a power of two that keeps it inside FP16's range;
  // 1 in the other forms and for the mask field (j = nch)
  float scale0[4], scale1[4];
  // 1: in the BF16 and FP16 forms the z pass runs the forward z-axis DFT of
  // the channel fields on the tensor cores (k_zmac_tc) where its length allows
  int tc;
  // set to 1 by a tensor-core pass whose bounded wait for its own MMAs ran out
  // (it then stops and returns); nullptr: not reported
  int* tc_err;
  // X of the tensor-core z pass, [r][kx <= Px/2][ky][kz] per launch group
  // (the handle allocates it with the tensor-core forms); nullptr: the z pass
  // runs as one kernel
  float2* zx;
};

constexpr int kStoreF32 = 0, kStoreBF16 = 1, kStoreF16 = 2;

// a[j] for a field index j known only at run time, without indexing the
// kernel-parameter array (which would copy it to local memory)
__device__ __forceinline__ float field_scale(const float (&a)[4], int j) {
  return j == 0 ? a[0] : j == 1 ? a[1] : j == 2 ? a[2] : a[3];
}

// Storage of the packed fields of F0 / F1 for a batch of rotations: the
// channel fields j < nch hold FP32 complex values, or 16-bit pairs in the
// reduced-precision forms (BF16; FP16 with a per-field power-of-two scale);
// the mask field j = nch is always FP32 complex, so the overlap count N(chi)
// keeps FP32 accuracy.  E = complex values per field.  put and get take and
// return the field's true values; the FP16 scale is applied inside.
template <int ST>
struct Fields {
  static constexpr int CB = ST == kStoreF32 ? 8 : 4;   // bytes per channel-field value
  __host__ __device__ static long long rot_bytes(const Geo& g, long long E) {
    return (long long)g.nch * E * CB + E * 8;
  }
  __device__ __forceinline__ static char* field(void* base, const Geo& g, long long E, int r, int j) {
    return (char*)base + (long long)r * rot_bytes(g, E) + (long long)j * E * CB;
  }
  __device__ __forceinline__ static const char* field(const void* base, const Geo& g, long long E,
                                                      int r, int j) {
    return (const char*)base + (long long)r * rot_bytes(g, E) + (long long)j * E * CB;
  }
  // scale: the field's storage scale (FP16 form; ignored otherwise)
  __device__ __forceinline__ static void put(char* f, long long i, float2 v, bool mask, float scale) {
    if (ST == kStoreBF16 && !mask) reinterpret_cast<__nv_bfloat162*>(f)[i] = __float22bfloat162_rn(v);
    else if (ST == kStoreF16 && !mask)
      reinterpret_cast<__half2*>(f)[i] = __float22half2_rn(make_float2(v.x * scale, v.y * scale));
    else reinterpret_cast<float2*>(f)[i] = v;
  }
  // inv_scale: 1 / the field's storage scale (FP16 form; ignored otherwise)
  __device__ __forceinline__ static float2 get(const char* f, long long i, bool mask, float inv_scale) {
    if (ST == kStoreBF16 && !mask) return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(f)[i]);
    if (ST == kStoreF16 && !mask) {
      const float2 v = __half22float2(reinterpret_cast<const __half2*>(f)[i]);
      return make_float2(v.x * inv_scale, v.y * inv_scale);
    }
    return reinterpret_cast<const float2*>(f)[i];
  }
};

// per-rotation matrix (row-major, acts on (x, y, z)), rounded to FP32 on the host
struct RotMat { float m[9]; };

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// orderable key: larger score -> larger key; equal score -> smaller index wins
__device__ __forceinline__ unsigned long long make_key(float s, unsigned lin) {
  unsigned u = __float_as_uint(s);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 32) | (unsigned long long)(0xFFFFFFFFu - lin);
}

// ----------------------------------------------------------------- resample
// Section 3.2: B_hat(x) = B(R (x - c) + c), trilinear; the rotated mask is
// [trilinear M_B >= 0.5] inside [0, n-1]^3 (+-1e-4).  The sample point and the
// mask decision use round-to-nearest FP32 operations in a fixed order (no
// contraction), so the decision is reproducible bit for bit.  B and M_B are
// read as the row-pair table and corner codes k_pack_floating prepares (BQ,
// C8: nvox entries each).
__global__ void k_pack_floating(const float* __restrict__ B, const uint8_t* __restrict__ MB, Geo g,
                                float4* __restrict__ BQ, uint8_t* __restrict__ C8);
__global__ void k_resample(const float4* __restrict__ BQ, const uint8_t* __restrict__ C8,
                           const RotMat* __restrict__ rot, Geo g, float* __restrict__ Bh,
                           uint8_t* __restrict__ Mh, int* __restrict__ msum, int* __restrict__ marg);
// The rotated masks alone, counted into msum and marg as k_resample counts
// them (the same decisions from the same corner codes, no volumes written):
// the pre-pass that bounds the shifts of a whole call.  Grid: resample_grid.
__global__ void k_mask_counts(const uint8_t* __restrict__ C8, const RotMat* __restrict__ rot, Geo g,
                              int* __restrict__ msum, int* __restrict__ marg);
constexpr int kResampleZGroups = 8;            // z-plane groups of 4 per resample block
inline dim3 resample_grid(const Geo& g, int nrot) {
  return dim3((unsigned)((g.nx + 7) / 8), (unsigned)((g.ny + 3) / 4),
              (unsigned)(((g.nz + 4 * kResampleZGroups - 1) / (4 * kResampleZGroups)) * nrot));
}

// ----------------------------------------------------------------- shift bounds
// Marginal mask counts per axis, [nz | ny | nx] per volume (marg in k_resample
// fills them for each rotated mask; k_marginals for the fixed mask).  For a
// shift chi, N(chi) <= sum_i min(a_i, b_{i + chi_axis}) over the slabs of any
// axis, so shifts whose slab bound is below the Section 3.2 overlap threshold
// are invalid; k_shift_bounds keeps, per rotation and axis, the range of shift
// slots that can be valid ([lo, hi] in v = chi + n - 1; lo > hi: none).
__global__ void k_marginals(const uint8_t* __restrict__ M, Geo g, int* __restrict__ marg);
__global__ void k_shift_bounds(const int* __restrict__ margA, const int* __restrict__ margB,
                               const int* __restrict__ msumB, int sumA, float gamma, Geo g,
                               int* __restrict__ bounds);
__global__ void k_fill(float* __restrict__ p, long long n, float v);
// results scored in a regrouped order back to the caller's: entry i belongs
// to rotation perm[i]
__global__ void k_scatter_results(const int* __restrict__ perm, const float* __restrict__ score,
                                  const int32_t* __restrict__ shift, int n,
                                  float* __restrict__ out_score, int32_t* __restrict__ out_shift);

// sum of a uint8 mask (for the fixed volume)
__global__ void k_mask_sum(const uint8_t* __restrict__ M, long long n, int* __restrict__ out);

// per-rotation overlap threshold in FFT units: (max(1, ceil(gamma min(sA, sB))) - 0.5) * Pz Py Px
__global__ void k_thresholds(const int* __restrict__ msumB, int sumA, float gamma, double pvol,
                             int nrot, float* __restrict__ thr);

// decode per-rotation keys into (score, shift)
__global__ void k_finalize(const unsigned long long* __restrict__ keys, int nrot, Geo g,
                           float* __restrict__ best_score, int32_t* __restrict__ best_shift);

// copy a float volume / mask into the rotation-0 slot (fixed-volume prepare)
__global__ void k_copy_in(const float* __restrict__ A, const uint8_t* __restrict__ MA,
                          long long n, float* __restrict__ Bh, uint8_t* __restrict__ Mh);

// ----------------------------------------------------------------- FFT passes
// F0 / F1 are laid out by Fields<g.store> (FP32 everywhere when g.store == kStoreF32).
// v: split variant of the length P (SplitV<P, v>; 0 = the built-in one, 1 =
// the alternative where P has one, chosen by the autotuner)
template <int P> void launch_fwd_x(const float* Bh, const uint8_t* Mh, void* F0, const float2* tw,
                                   Geo g, int nrot, cudaStream_t st, int v = 0);
template <int P> void launch_fwd_y(const void* F0, void* F1, const float2* tw, Geo g, int nrot,
                                   cudaStream_t st, int v = 0);
template <int P> void launch_zmac(const void* F1, const float2* UV, float2* F2, const float2* tw,
                                  Geo g, int nrot, const int* bounds, cudaStream_t st, int v = 0);
template <int P> void launch_prep_z(const float2* F1, float2* UV, const float2* tw, Geo g,
                                    cudaStream_t st);
template <int P> void launch_inv_y(const float2* F2, float2* F3, const float2* tw, Geo g, int nrot,
                                   const int* bounds, cudaStream_t st, int v = 0);
template <int P> void launch_inv_x(const float2* F3, const float* thr, unsigned long long* keys,
                                   float* map, const float2* tw, Geo g, int nrot, const int* bounds,
                                   cudaStream_t st, int v = 0);
// bounds: per rotation {lo_z, hi_z, lo_y, hi_y, lo_x, hi_x} shift slots that can
// be valid, or nullptr for the full range

}  // namespace csngf
