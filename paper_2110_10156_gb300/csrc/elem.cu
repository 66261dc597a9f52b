// Element-wise kernels: trilinear rotate-resample with the rotated mask
// (Section 3.2), mask sums, overlap thresholds and result decoding.
#include "kernels.cuh"

namespace csngf {

namespace {
struct AxisSample {
  bool inside;
  int i0;
  float t;
};

// domain test, clamped base index and fraction for one axis (FP32, no contraction)
__device__ __forceinline__ AxisSample axis_sample(float p, int n) {
  AxisSample a;
  const float slack = 1e-4f;
  const float hi = __fadd_rn((float)(n - 1), slack);
  a.inside = (p >= -slack) && (p <= hi);
  float pc = fminf(fmaxf(p, 0.0f), (float)(n - 1));
  int i0 = (int)floorf(pc);
  i0 = min(i0, n - 2);
  a.i0 = i0;
  a.t = __fsub_rn(pc, (float)i0);
  return a;
}

// (1 - t) a + t b as two fused multiply-adds: a at t = 0, b at t = 1 exactly
__device__ __forceinline__ float lerp_exact(float a, float b, float t) {
  return fmaf(t, b, fmaf(-t, a, a));
}

__device__ __forceinline__ float lerp_rn(float a, float b, float t) {
  return __fadd_rn(a, __fmul_rn(t, __fsub_rn(b, a)));
}
}  // namespace

// The floating volume as the resample reads it, prepared once per call and
// shared by every rotation: BQ[i] = (B[i], B[i+1], B[i+sy], B[i+sy+1]), the
// x-pairs of rows y and y+1, so the four corners of a cell's z-face come in
// one 16-byte load (one sector instead of two), and corner codes C8[i] whose
// bit k is M_B at corner (dx, dy, dz) = (k & 1, (k >> 1) & 1, k >> 2) of the
// cell with base voxel i, so the eight mask corners come in one byte.  A cell
// base is never on a far face (axis_sample clamps i0 <= n - 2); entries past
// the volume hold 0.
__global__ void k_pack_floating(const float* __restrict__ B, const uint8_t* __restrict__ MB, Geo g,
                                float4* __restrict__ BQ, uint8_t* __restrict__ C8) {
  const int sy = g.nx, sz = g.nx * g.ny;          // volumes hold < 2^31 voxels
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.nvox;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / sz);
    const bool in_x = x + 1 < g.nx, in_y = y + 1 < g.ny;
    BQ[i] = make_float4(B[i], in_x ? B[i + 1] : 0.0f, in_y ? B[i + sy] : 0.0f,
                        in_x && in_y ? B[i + sy + 1] : 0.0f);
    unsigned bits = 0;
    if (in_x && y + 1 < g.ny && z + 1 < g.nz) {
      const int o[8] = {0, 1, sy, sy + 1, sz, sz + 1, sz + sy, sz + sy + 1};
#pragma unroll
      for (int k = 0; k < 8; ++k) bits |= (MB[i + o[k]] ? 1u : 0u) << k;
    }
    C8[i] = (uint8_t)bits;
  }
}

// The sample point p = R (x - c) + c of voxel (x, y, z), per axis
// ((R0 dx + R1 dy) + R2 dz) + c in round-to-nearest FP32 without contraction.
// A resample thread keeps x and y over its z-planes, so the first sum is
// formed once per thread (SampleRow) and each plane adds its z term in the
// same order: the same floats as forming the whole sum per voxel.
struct SampleRow {
  float s[3];                                   // rn(rn(R_i0 dx) + rn(R_i1 dy))
};
__device__ __forceinline__ SampleRow sample_row(const RotMat& R, const Geo& g, int x, int y) {
  const float cx = 0.5f * (float)(g.nx - 1), cy = 0.5f * (float)(g.ny - 1);
  const float dx = __fsub_rn((float)x, cx), dy = __fsub_rn((float)y, cy);
  SampleRow sr;
#pragma unroll
  for (int i = 0; i < 3; ++i) sr.s[i] = __fadd_rn(__fmul_rn(R.m[3 * i + 0], dx), __fmul_rn(R.m[3 * i + 1], dy));
  return sr;
}
__device__ __forceinline__ void sample_axes(const RotMat& R, const SampleRow& sr, const Geo& g, int z,
                                            AxisSample& ax, AxisSample& ay, AxisSample& az) {
  const float cx = 0.5f * (float)(g.nx - 1), cy = 0.5f * (float)(g.ny - 1),
              cz = 0.5f * (float)(g.nz - 1);
  const float dz = __fsub_rn((float)z, cz);
  float p[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    p[i] = __fadd_rn(__fadd_rn(sr.s[i], __fmul_rn(R.m[3 * i + 2], dz)), i == 0 ? cx : (i == 1 ? cy : cz));
  ax = axis_sample(p[0], g.nx);
  ay = axis_sample(p[1], g.ny);
  az = axis_sample(p[2], g.nz);
}

// the mask decision [trilinear M_B >= 0.5] from the cell's corner code: lerps
// along x, y, z in round-to-nearest FP32 with no contraction; when the eight
// corners agree every lerp a + t (a - a) returns a exactly
__device__ __forceinline__ uint8_t mask_decision(unsigned bits, float tx, float ty, float tz) {
  if (bits == 0u) return 0;
  if (bits == 0xffu) return 1;
  float c[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) c[k] = ((bits >> k) & 1u) ? 1.0f : 0.0f;
  const float m00 = lerp_rn(c[0], c[1], tx), m01 = lerp_rn(c[2], c[3], tx);
  const float m10 = lerp_rn(c[4], c[5], tx), m11 = lerp_rn(c[6], c[7], tx);
  const float m0 = lerp_rn(m00, m01, ty), m1 = lerp_rn(m10, m11, ty);
  return lerp_rn(m0, m1, tz) >= 0.5f ? 1 : 0;
}

// the rotated mask alone: the same sample point and decision as resample_voxel
__device__ __forceinline__ uint8_t mask_voxel(const uint8_t* __restrict__ C8, const RotMat& R,
                                              const SampleRow& sr, const Geo& g, int z) {
  AxisSample ax, ay, az;
  sample_axes(R, sr, g, z, ax, ay, az);
  if (!(ax.inside && ay.inside && az.inside)) return 0;
  const int b000 = az.i0 * (g.nx * g.ny) + ay.i0 * g.nx + ax.i0;
  return mask_decision(__ldg(&C8[b000]), ax.t, ay.t, az.t);
}

__device__ __forceinline__ void resample_voxel(const float4* __restrict__ BQ,
                                               const uint8_t* __restrict__ C8, const RotMat& R,
                                               const SampleRow& sr, const Geo& g, int z, float& val,
                                               uint8_t& m) {
  AxisSample ax, ay, az;
  sample_axes(R, sr, g, z, ax, ay, az);
  val = 0.0f;
  m = 0;
  if (ax.inside && ay.inside && az.inside) {
    const int sy = g.nx, sz = g.nx * g.ny;        // volumes hold < 2^31 voxels
    const int b000 = az.i0 * sz + ay.i0 * sy + ax.i0;
    const float4 q0 = __ldg(&BQ[b000]), q1 = __ldg(&BQ[b000 + sz]);   // z-faces z0, z0 + 1
    const float2 c00 = make_float2(q0.x, q0.y), c01 = make_float2(q0.z, q0.w);
    const float2 c10 = make_float2(q1.x, q1.y), c11 = make_float2(q1.z, q1.w);
    const unsigned bits = __ldg(&C8[b000]);
    // intensity: lerps along x, y, z, exact at t = 0 and t = 1 so that
    // quarter turns reproduce the voxels bit for bit
    const float v00 = lerp_exact(c00.x, c00.y, ax.t), v01 = lerp_exact(c01.x, c01.y, ax.t);
    const float v10 = lerp_exact(c10.x, c10.y, ax.t), v11 = lerp_exact(c11.x, c11.y, ax.t);
    const float v0 = lerp_exact(v00, v01, ay.t), v1 = lerp_exact(v10, v11, ay.t);
    val = lerp_exact(v0, v1, az.t);
    m = mask_decision(bits, ax.t, ay.t, az.t);
  }
}

// Section 3.2 resample.  Block: 8 x 4 voxels per warp (x fastest), so one
// warp's sample points form a compact rotated 8 x 4 patch; four warps take
// four consecutive z-planes, and each thread repeats that for RZ plane groups
// (block: 8 x 4 x 4*RZ voxels).  Mask counts per axis (the slab bound's
// marginals) are reduced with warp shuffles before one atomic per slot.
// Grid: (x tiles, y tiles, z tiles * rotations).
// MONLY: only the rotated mask, counted (no volumes written)
template <bool MONLY>
__device__ __forceinline__ void resample_block(const float4* __restrict__ BQ,
                                               const uint8_t* __restrict__ C8,
                                               const RotMat* __restrict__ rot, const Geo& g,
                                               float* __restrict__ Bh, uint8_t* __restrict__ Mh,
                                               int* __restrict__ msum, int* __restrict__ marg) {
  constexpr int RZ = kResampleZGroups, ZB = 4 * RZ;    // z-planes per block
  const int ztiles = (g.nz + ZB - 1) / ZB;
  const int r = blockIdx.z / ztiles, zt = blockIdx.z - r * ztiles;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int tx = lane & 7, ty = lane >> 3;
  const int x = blockIdx.x * 8 + tx;
  const int y = blockIdx.y * 4 + ty;
  __shared__ int zs[ZB], ys[4][4], xs[4][8], cs[4];
  const RotMat R = rot[r];
  const SampleRow sr = sample_row(R, g, x, y);
  const bool xy_ok = x < g.nx && y < g.ny;
  const long long plane = (long long)g.nx * g.ny;
  // output index of plane z = zt*ZB + wid, advanced by four planes per group
  long long idx = (long long)r * g.nvox + (long long)(zt * ZB + wid) * plane + (long long)y * g.nx + x;
  int c = 0;                                   // this thread's mask voxels
#pragma unroll 1
  for (int k = 0; k < RZ; ++k, idx += 4 * plane) {
    const int z = zt * ZB + 4 * k + wid;
    int mk = 0;
    if (xy_ok && z < g.nz) {
      if constexpr (MONLY) {
        mk = mask_voxel(C8, R, sr, g, z);
      } else {
        float val;
        uint8_t m;
        resample_voxel(BQ, C8, R, sr, g, z, val, m);
        Bh[idx] = val;
        Mh[idx] = m;
        mk = m;
      }
    }
    c += mk;
    const int wz = __reduce_add_sync(0xffffffffu, mk);      // plane z, this warp's patch
    if (lane == 0) zs[4 * k + wid] = wz;
  }
  int cy = c;                                  // lanes sharing ty: xor over the tx bits
  cy += __shfl_xor_sync(0xffffffffu, cy, 1);
  cy += __shfl_xor_sync(0xffffffffu, cy, 2);
  cy += __shfl_xor_sync(0xffffffffu, cy, 4);
  int cx = c;                                  // lanes sharing tx: xor over the ty bits
  cx += __shfl_xor_sync(0xffffffffu, cx, 8);
  cx += __shfl_xor_sync(0xffffffffu, cx, 16);
  if (tx == 0) ys[wid][ty] = cy;
  if (ty == 0) xs[wid][tx] = cx;
  const int cw = __reduce_add_sync(0xffffffffu, c);
  if (lane == 0) cs[wid] = cw;
  __syncthreads();
  const int t = threadIdx.x;
  if (t == 0) {
    const int total = cs[0] + cs[1] + cs[2] + cs[3];
    if (total) atomicAdd(&msum[r], total);
  }
  if (marg) {
    int* mr = marg + (long long)r * (g.nz + g.ny + g.nx);
    if (t < ZB) {                              // z = zt*ZB + t (4k + wid = t)
      const int v = zs[t];
      if (v) atomicAdd(&mr[zt * ZB + t], v);
    } else if (t < ZB + 4) {
      const int q = t - ZB;
      const int v = ys[0][q] + ys[1][q] + ys[2][q] + ys[3][q];
      if (v) atomicAdd(&mr[g.nz + blockIdx.y * 4 + q], v);
    } else if (t < ZB + 12) {
      const int q = t - ZB - 4;
      const int v = xs[0][q] + xs[1][q] + xs[2][q] + xs[3][q];
      if (v) atomicAdd(&mr[g.nz + g.ny + blockIdx.x * 8 + q], v);
    }
  }
}

__global__ void __launch_bounds__(128)
k_resample(const float4* __restrict__ BQ, const uint8_t* __restrict__ C8,
           const RotMat* __restrict__ rot, Geo g, float* __restrict__ Bh, uint8_t* __restrict__ Mh,
           int* __restrict__ msum, int* __restrict__ marg) {
  resample_block<false>(BQ, C8, rot, g, Bh, Mh, msum, marg);
}

__global__ void __launch_bounds__(128)
k_mask_counts(const uint8_t* __restrict__ C8, const RotMat* __restrict__ rot, Geo g,
              int* __restrict__ msum, int* __restrict__ marg) {
  resample_block<true>(nullptr, C8, rot, g, nullptr, nullptr, msum, marg);
}

__global__ void k_marginals(const uint8_t* __restrict__ M, Geo g, int* __restrict__ marg) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.nvox;
       i += (long long)gridDim.x * blockDim.x) {
    if (!M[i]) continue;
    const int x = (int)(i % g.nx);
    const int y = (int)((i / g.nx) % g.ny);
    const int z = (int)(i / ((long long)g.nx * g.ny));
    atomicAdd(&marg[z], 1);
    atomicAdd(&marg[g.nz + y], 1);
    atomicAdd(&marg[g.nz + g.ny + x], 1);
  }
}

// block (rotation r, axis a); thread per shift slot v
__global__ void k_shift_bounds(const int* __restrict__ margA, const int* __restrict__ margB,
                               const int* __restrict__ msumB, int sumA, float gamma, Geo g,
                               int* __restrict__ bounds) {
  const int r = blockIdx.x, a = blockIdx.y;
  const int n = a == 0 ? g.nz : (a == 1 ? g.ny : g.nx);
  const int off = a == 0 ? 0 : (a == 1 ? g.nz : g.nz + g.ny);
  const int* ma = margA + off;
  const int* mb = margB + (long long)r * (g.nz + g.ny + g.nx) + off;
  const int mn = min(sumA, msumB[r]);
  double t = ceil((double)gamma * (double)mn);
  if (t < 1.0) t = 1.0;
  const long long thr = (long long)t;
  __shared__ int lo_s, hi_s;
  if (threadIdx.x == 0) { lo_s = 0x7fffffff; hi_s = -1; }
  __syncthreads();
  for (int v = threadIdx.x; v < 2 * n - 1; v += blockDim.x) {
    const int c = v - (n - 1);
    long long u = 0;
    for (int i = max(0, -c); i < min(n, n - c); ++i) u += min(ma[i], mb[i + c]);
    if (u >= thr) {
      atomicMin(&lo_s, v);
      atomicMax(&hi_s, v);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bounds[r * 6 + 2 * a] = lo_s;
    bounds[r * 6 + 2 * a + 1] = hi_s;
  }
}

__global__ void k_scatter_results(const int* __restrict__ perm, const float* __restrict__ score,
                                  const int32_t* __restrict__ shift, int n,
                                  float* __restrict__ out_score, int32_t* __restrict__ out_shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = perm[i];
  out_score[r] = score[i];
#pragma unroll
  for (int a = 0; a < 3; ++a) out_shift[3 * (long long)r + a] = shift[3 * (long long)i + a];
}

__global__ void k_fill(float* __restrict__ p, long long n, float v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_mask_sum(const uint8_t* __restrict__ M, long long n, int* __restrict__ out) {
  int c = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    c += M[i] ? 1 : 0;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void k_thresholds(const int* __restrict__ msumB, int sumA, float gamma, double pvol,
                             int nrot, float* __restrict__ thr) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrot) return;
  const int mn = min(sumA, msumB[r]);
  double t = ceil((double)gamma * (double)mn);
  if (t < 1.0) t = 1.0;
  thr[r] = (float)((t - 0.5) * pvol);
}

__global__ void k_finalize(const unsigned long long* __restrict__ keys, int nrot, Geo g,
                           float* __restrict__ best_score, int32_t* __restrict__ best_shift) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrot) return;
  const unsigned long long k = keys[r];
  if (k == 0ull) {
    best_score[r] = __int_as_float(0xff800000);   // -inf: no valid shift
    best_shift[3 * r + 0] = 0;
    best_shift[3 * r + 1] = 0;
    best_shift[3 * r + 2] = 0;
    return;
  }
  unsigned u = (unsigned)(k >> 32);
  u = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  const unsigned lin = 0xFFFFFFFFu - (unsigned)(k & 0xFFFFFFFFull);
  const int vx = (int)(lin % (unsigned)g.vx);
  const int vy = (int)((lin / (unsigned)g.vx) % (unsigned)g.vy);
  const int vz = (int)(lin / ((unsigned)g.vx * (unsigned)g.vy));
  best_score[r] = __uint_as_float(u);
  best_shift[3 * r + 0] = vz - (g.nz - 1);
  best_shift[3 * r + 1] = vy - (g.ny - 1);
  best_shift[3 * r + 2] = vx - (g.nx - 1);
}

__global__ void k_copy_in(const float* __restrict__ A, const uint8_t* __restrict__ MA, long long n,
                          float* __restrict__ Bh, uint8_t* __restrict__ Mh) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    Bh[i] = A[i];
    Mh[i] = MA[i] ? 1 : 0;
  }
}

}  // namespace csngf
