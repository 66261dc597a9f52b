// FFT passes of the all-shift NGF correlation (Cross-Sim-NGF Eq. 6-8).
// Included by one translation unit per FFT length (passes_<P>.cu).
#pragma once

#include "kernels.cuh"

namespace csngf {

// Output index m of a length-P circular correlation -> the shift slot
// v = chi + n - 1 in [lo, hi] with chi = m or chi = m - P, or -1 if neither
// lies there.  Slot m sums the linear correlation at every chi = m (mod P);
// it equals the value at the one chi in [lo, hi] when every other chi of that
// class lies outside the linear support [-(n-1), n-1], which the caller
// guarantees by P >= n + max(n-1-lo, hi-(n-1)) (with lo = 0, hi = 2n-2 that
// is the full linear-correlation length P >= 2n-1).
__device__ __forceinline__ int shift_slot(int m, int n, int P, int lo, int hi) {
  const int v1 = m + n - 1;                      // chi = m
  if (m <= n - 1 && v1 >= lo && v1 <= hi) return v1;
  const int v2 = m - P + n - 1;                  // chi = m - P
  if (v2 >= 0 && v2 >= lo && v2 <= hi) return v2;
  return -1;
}

// Forward-transform inputs: a volume side n is zero padded to P.  When
// n <= P/2 the upper half of every step-1 sequence is zero and step 1 is the
// pruned form (FourStep::step1_half); otherwise all N1 inputs are read.
template <class FS, bool HALF>
struct FwdIn {
  static constexpr int NI = HALF ? FS::N1 / 2 : FS::N1;   // step-1 inputs per thread
  template <int S, bool TS = false>
  __device__ __forceinline__ static void step1(float2 (&v)[NI], float2* ex_seq, int n2,
                                               const float2* __restrict__ twN) {
    if constexpr (HALF) FS::template step1_half<S, TS>(v, ex_seq, n2, twN);
    else FS::template step1<S, TS>(v, ex_seq, n2, twN);
  }
};

// calls f with the storage form of the channel fields as a compile-time constant
template <class F>
static void by_store(int store, F&& f) {
  if (store == kStoreBF16) f(std::integral_constant<int, kStoreBF16>{});
  else if (store == kStoreF16) f(std::integral_constant<int, kStoreF16>{});
  else f(std::integral_constant<int, kStoreF32>{});
}

// calls f with split variant v of length P (0 where P has no second split)
template <int P, class F>
static void by_split(int v, F&& f) {
  if constexpr (has_alt_split(P)) {
    if (v == 1) {
      f(std::integral_constant<int, 1>{});
      return;
    }
  }
  f(std::integral_constant<int, 0>{});
}

template <class K>
static void set_smem(K kern, size_t bytes) {
  if (bytes > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ---------------------------------------------------------------------------
// fwd_x: Eq. 1 NGF of the resampled volume, the Eq. 6 channels packed in four
// complex fields, and the x-axis FFT of every row (zero padded to Px).
// Block: ROWS rows of one slab; thread (row, n2) gathers x = N2*n1 + n2.
// ---------------------------------------------------------------------------
// A thread keeps the NGF (x, y, z, mask) of its step-1 inputs across the
// four fields: in registers for half-length inputs, in its own slots of
// shared memory [NI][NT] (float4) for full-length ones, which would spill.
template <int P, bool HALF, int V>
struct FwdXCfg {
  static constexpr int N2 = SplitV<P, V>::N2;
  static constexpr int ROWS = (256 / N2) > 0 ? (256 / N2) : 1;
  static constexpr int NT = ROWS * N2;
  static constexpr int NI = FwdIn<FourStep<P, true, V>, HALF>::NI;
  static constexpr size_t ex_bytes = ((size_t)ROWS * FourStep<P, true, V>::CS * sizeof(float2) + 15) / 16 * 16;
  static constexpr size_t smem_bytes = ex_bytes + (HALF ? 0 : (size_t)NI * NT * sizeof(float4));
  // three blocks per SM (at most 80 registers per thread): the gradient
  // gathers and the per-field barriers leave the pass latency-bound, and the
  // extra resident warps hide more of it than the few spilled registers cost
  // (measured: 200-point lengths 2.13 -> 1.67 ms per 32 rotations, 320-point
  // half-input lengths 72 -> 65 ms per 1000 rotations; 400 and 320 unchanged)
  static constexpr int MIN_BLOCKS = 3;
};

template <int P, int ROWS, int ST, bool HALF, int V>
__global__ void __launch_bounds__(ROWS * SplitV<P, V>::N2, FwdXCfg<P, HALF, V>::MIN_BLOCKS)
k_fwd_x(const float* __restrict__ Bh, const uint8_t* __restrict__ Mh, void* __restrict__ F0,
        const float2* __restrict__ tw, Geo g, long long nrows) {
  using FS = FourStep<P, true, V>;
  using FI = FwdIn<FS, HALF>;
  constexpr int N1 = FS::N1, N2 = FS::N2, CS = FS::CS, H = FI::NI;
  extern __shared__ float2 ex[];
  const int t = threadIdx.x;
  const int lrow = t / N2, n2 = t - lrow * N2;
  const long long grow = (long long)blockIdx.x * ROWS + lrow;
  const bool row_ok = grow < nrows;
  const long long rz = row_ok ? grow / g.ny : 0;
  const int y = row_ok ? (int)(grow - rz * g.ny) : 0;
  const int r = (int)(rz / g.nz), z = (int)(rz - (long long)r * g.nz);

  // x = N2*n1 + n2 < nx: with nx <= P/2 only n1 < N1/2 can hold data
  constexpr bool NS = !HALF;                  // NGF staged in shared memory
  constexpr int HR = NS ? 1 : H;
  float vx[HR], vy[HR], vz[HR], mm[HR];
  float4* ngs = reinterpret_cast<float4*>(reinterpret_cast<char*>(ex) + FwdXCfg<P, HALF, V>::ex_bytes);
  const int NTX = ROWS * N2;
  const float* Vol = Bh + (long long)r * g.nvox;
  const uint8_t* M = Mh + (long long)r * g.nvox;
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  const int ym = max(y - 1, 0), yp = min(y + 1, g.ny - 1);
  const int zm = max(z - 1, 0), zp = min(z + 1, g.nz - 1);
  const long long base = (long long)z * sz + (long long)y * sy;
  const long long rows_per_field = (long long)g.nz * g.ny;
  const int nrot = (int)(nrows / rows_per_field);
  const bool has_partner = !(r & 1) && r + 1 < nrot;
  // per element: the NGF times the mask (m^2 = m, so every Eq. 6 product of
  // two masked components equals the product times m, bit for bit) and the
  // mask pair of the mask field coded as m + 2 m2 (m2: the next rotation's mask)
#pragma unroll
  for (int n1 = 0; n1 < H; ++n1) {
    const int x = N2 * n1 + n2;
    float4 q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (row_ok && x < g.nx) {
      const int xm = max(x - 1, 0), xp = min(x + 1, g.nx - 1);
      const float gx = 0.5f * (__ldg(&Vol[base + xp]) - __ldg(&Vol[base + xm]));
      const float gy = 0.5f * (__ldg(&Vol[(long long)z * sz + (long long)yp * sy + x]) -
                               __ldg(&Vol[(long long)z * sz + (long long)ym * sy + x]));
      const float gz = 0.5f * (__ldg(&Vol[(long long)zp * sz + (long long)y * sy + x]) -
                               __ldg(&Vol[(long long)zm * sz + (long long)y * sy + x]));
      const float inv = rsqrtf(gx * gx + gy * gy + gz * gz + g.eps2);
      const float m = M[base + x] ? 1.0f : 0.0f;
      const float m2 = (has_partner && M[g.nvox + base + x]) ? 2.0f : 0.0f;
      q = make_float4(m * (gx * inv), m * (gy * inv), m * (gz * inv), m + m2);
    }
    if constexpr (NS) {
      ngs[n1 * NTX + t] = q;
    } else {
      vx[n1] = q.x;
      vy[n1] = q.y;
      vz[n1] = q.z;
      mm[n1] = q.w;
    }
  }
  // Masks are paired across consecutive rotations: the even rotation's mask
  // field carries (M_r, M_{r+1}); an odd rotation has no mask field of its own.
  const bool odd_block = ((blockIdx.x * (long long)ROWS) / rows_per_field & 1) &&
                         (blockIdx.x * (long long)ROWS) / rows_per_field ==
                             (min(blockIdx.x * (long long)ROWS + ROWS, nrows) - 1) / rows_per_field;
#pragma unroll 1
  for (int j = 0; j < g.nf; ++j) {
    if (j == g.nch && odd_block) break;          // uniform over the block
    // Eq. 6 products (squared measure) or Eq. 3 components (unsquared); the
    // mask field comes last
    const int code = j == g.nch ? 3 : (g.nch == 3 ? j : 4 + j);
    float2 v[H];
    // this field's inputs, with the field's product chosen at compile time
    auto inputs = [&](auto cc) {
      constexpr int CODE = decltype(cc)::value;
#pragma unroll
      for (int n1 = 0; n1 < H; ++n1) {
        float X, Y, Z, w;
        if constexpr (NS) {
          const float4 q = ngs[n1 * NTX + t];   // this thread's own slot
          X = q.x; Y = q.y; Z = q.z; w = q.w;
        } else {
          X = vx[n1 < HR ? n1 : 0]; Y = vy[n1 < HR ? n1 : 0]; Z = vz[n1 < HR ? n1 : 0];
          w = mm[n1 < HR ? n1 : 0];
        }
        if constexpr (CODE == 0) v[n1] = make_float2(X * X, Y * Y);
        else if constexpr (CODE == 1) v[n1] = make_float2(Z * Z, X * Y);
        else if constexpr (CODE == 2) v[n1] = make_float2(X * Z, Y * Z);
        else if constexpr (CODE == 4) v[n1] = make_float2(X, Y);
        else if constexpr (CODE == 5) v[n1] = make_float2(Z, 0.0f);
        else {                                   // mask pair (M_r, M_{r+1}); w = m + 2 m2
          const float m2 = w >= 2.0f ? 1.0f : 0.0f;
          v[n1] = (r & 1) ? make_float2(0.0f, 0.0f) : make_float2(w - 2.0f * m2, m2);
        }
      }
    };
    switch (code) {
      case 0: inputs(std::integral_constant<int, 0>{}); break;
      case 1: inputs(std::integral_constant<int, 1>{}); break;
      case 2: inputs(std::integral_constant<int, 2>{}); break;
      case 4: inputs(std::integral_constant<int, 4>{}); break;
      case 5: inputs(std::integral_constant<int, 5>{}); break;
      default: inputs(std::integral_constant<int, 3>{}); break;
    }
    FI::template step1<-1>(v, ex + lrow * CS, n2, tw);
    __syncthreads();
    if (t < ROWS * N1) {
      const int lr = t / N1, k1 = t - lr * N1;
      const long long gr = (long long)blockIdx.x * ROWS + lr;
      const bool skip_row = j == g.nch && ((gr / rows_per_field) & 1);   // odd rotation: no mask field
      if (gr < nrows && !skip_row) {
        float2 u[N2];
        FS::template step2<-1>(u, ex + lr * CS, k1);
        const long long rz2 = gr / g.ny;
        const int y2 = (int)(gr - rz2 * g.ny);
        const int r2 = (int)(rz2 / g.nz), z2 = (int)(rz2 - (long long)r2 * g.nz);
        char* fld = Fields<ST>::field(F0, g, rows_per_field * P, r2, j);
        const long long row = ((long long)z2 * g.ny + y2) * P;
        const float sc = field_scale(g.scale0, j);
        if (j == g.nch) {
#pragma unroll
          for (int k2 = 0; k2 < N2; ++k2) Fields<ST>::put(fld, row + k1 + N1 * k2, u[k2], true, sc);
        } else {
#pragma unroll
          for (int k2 = 0; k2 < N2; ++k2) Fields<ST>::put(fld, row + k1 + N1 * k2, u[k2], false, sc);
        }
      }
    }
    __syncthreads();
  }
}

template <int P, bool HALF, int V>
void launch_fwd_x_t(const float* Bh, const uint8_t* Mh, void* F0, const float2* tw, Geo g, int nrot,
                    cudaStream_t st) {
  constexpr int N2 = SplitV<P, V>::N2;
  constexpr int ROWS = FwdXCfg<P, HALF, V>::ROWS;
  const long long nrows = (long long)nrot * g.nz * g.ny;
  const size_t smem = FwdXCfg<P, HALF, V>::smem_bytes;
  const unsigned blocks = (unsigned)((nrows + ROWS - 1) / ROWS);
  auto go = [&](auto kern) {
    set_smem(kern, smem);
    kern<<<blocks, ROWS * N2, smem, st>>>(Bh, Mh, F0, tw, g, nrows);
  };
  by_store(g.store, [&](auto st) { go(k_fwd_x<P, ROWS, decltype(st)::value, HALF, V>); });
}

template <int P>
void launch_fwd_x(const float* Bh, const uint8_t* Mh, void* F0, const float2* tw, Geo g, int nrot,
                  cudaStream_t st, int v) {
  by_split<P>(v, [&](auto vc) {
    constexpr int V = decltype(vc)::value;
    if (2 * g.nx <= P) launch_fwd_x_t<P, true, V>(Bh, Mh, F0, tw, g, nrot, st);
    else launch_fwd_x_t<P, false, V>(Bh, Mh, F0, tw, g, nrot, st);
  });
}

// ---------------------------------------------------------------------------
// fwd_y: y-axis FFT of every column of F0 (rows y >= ny are zero); the output
// is transposed so that ky is contiguous for the z pass.
// Block: W consecutive kx of one (r, j, z) plane.
// ---------------------------------------------------------------------------
// Blocks per SM for the single-transform passes: as many as keep at least
// MINR registers per thread (each of the SM's four sub-partitions holds 16384
// registers for the warps placed on it) and fit in shared memory.
constexpr int pass_blocks(int threads, size_t smem, int minr) {
  int best = 1;
  for (int b = 2; b <= 8; ++b) {
    const int per_sub = (b * ((threads + 31) / 32) + 3) / 4;
    const int regs = (16384 / (32 * per_sub)) / 8 * 8;
    if (regs >= minr && (size_t)b * (smem + 1024) <= 228 * 1024) best = b;
  }
  return best;
}
template <int P, int V> struct FwdYCfg {
  // 16 columns per block; 8 where the second stage is longer than 20 points
  // (more registers per thread: smaller blocks keep several per SM)
  static constexpr int W = SplitV<P, V>::N2 > 20 ? 8 : 16;
  static constexpr int NT = W * SplitV<P, V>::N2;
  static constexpr size_t smem_bytes = (size_t)W * FourStep<P, true, V>::CS * sizeof(float2);
  // the 25- and 32-point second stages need more registers than 16- or 20-point ones
  static constexpr int MIN_BLOCKS = pass_blocks(NT, smem_bytes, SplitV<P, V>::N2 > 20 ? 80 : 48);
};

template <int P, int W, int ST, bool HALF, int V>
__global__ void __launch_bounds__(W * SplitV<P, V>::N2, FwdYCfg<P, V>::MIN_BLOCKS)
k_fwd_y(const void* __restrict__ F0, void* __restrict__ F1, const float2* __restrict__ tw,
        Geo g) {
  using FS = FourStep<P, true, V>;
  using FI = FwdIn<FS, HALF>;
  constexpr int N1 = FS::N1, N2 = FS::N2, CS = FS::CS;
  extern __shared__ float2 ex[];
  const int t = threadIdx.x;
  // kx tiles run fastest over the grid, so the blocks that read the two halves
  // of a 128-byte line of F0 run together and the second one hits in L2
  const long long plane = blockIdx.y;                // ((r * nf) + j) * nz + z
  const long long rj = plane / g.nz;
  const int z = (int)(plane - rj * g.nz);
  const int r = (int)(rj / g.nf), j = (int)(rj - (long long)r * g.nf);
  const bool is_mask = j == g.nch;
  if (is_mask && (r & 1)) return;                    // paired into the even rotation's mask field
  const int kx0 = blockIdx.x * W;
  {
    const int col = t % W, n2 = t / W;
    const int kx = kx0 + col;
    const char* src = Fields<ST>::field(F0, g, (long long)g.nz * g.ny * g.Px, r, j);
    const float isc = 1.0f / field_scale(g.scale0, j);
    const long long zoff = (long long)z * g.ny * g.Px;
    float2 v[FI::NI];                     // y < ny: with ny <= P/2 the upper half is zero
    if (is_mask) {
#pragma unroll
      for (int n1 = 0; n1 < FI::NI; ++n1) {
        const int y = N2 * n1 + n2;
        v[n1] = (y < g.ny && kx < g.Px) ? Fields<ST>::get(src, zoff + (long long)y * g.Px + kx, true, isc)
                                        : make_float2(0.f, 0.f);
      }
    } else {
#pragma unroll
      for (int n1 = 0; n1 < FI::NI; ++n1) {
        const int y = N2 * n1 + n2;
        v[n1] = (y < g.ny && kx < g.Px) ? Fields<ST>::get(src, zoff + (long long)y * g.Px + kx, false, isc)
                                        : make_float2(0.f, 0.f);
      }
    }
    FI::template step1<-1>(v, ex + col * CS, n2, tw);
  }
  __syncthreads();
  if (t < W * N1) {
    const int col = t / N1, k1 = t - col * N1;
    const int kx = kx0 + col;
    if (kx < g.Px) {
      float2 u[N2];
      FS::template step2<-1>(u, ex + col * CS, k1);
      char* dst = Fields<ST>::field(F1, g, (long long)g.nz * g.Px * P, r, j);
      const long long row = ((long long)kx * g.nz + z) * P;       // [kx][z][ky]
      const float sc = field_scale(g.scale1, j);
      if (is_mask) {
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) Fields<ST>::put(dst, row + k1 + N1 * k2, u[k2], true, sc);
      } else {
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) Fields<ST>::put(dst, row + k1 + N1 * k2, u[k2], false, sc);
      }
    }
  }
}

template <int P, int V>
void launch_fwd_y_t(const void* F0, void* F1, const float2* tw, Geo g, int nrot, cudaStream_t st) {
  constexpr int W = FwdYCfg<P, V>::W, N2 = SplitV<P, V>::N2;
  const size_t smem = FwdYCfg<P, V>::smem_bytes;
  dim3 grid((unsigned)((g.Px + W - 1) / W), (unsigned)(nrot * g.nf * g.nz));   // y: at most 32 * 4 * 256
  auto go = [&](auto kern) {
    set_smem(kern, smem);
    kern<<<grid, W * N2, smem, st>>>(F0, F1, tw, g);
  };
  const bool half = 2 * g.ny <= P;
  by_store(g.store, [&](auto sf) {
    constexpr int ST = decltype(sf)::value;
    half ? go(k_fwd_y<P, W, ST, true, V>) : go(k_fwd_y<P, W, ST, false, V>);
  });
}

template <int P>
void launch_fwd_y(const void* F0, void* F1, const float2* tw, Geo g, int nrot, cudaStream_t st, int v) {
  by_split<P>(v, [&](auto vc) { launch_fwd_y_t<P, decltype(vc)::value>(F0, F1, tw, g, nrot, st); });
}

// ---------------------------------------------------------------------------
// zmac: for W columns (kx, ky) and their mirrors (-kx, -ky):
//   z-axis FFT of the four packed fields,
//   X(k) = sum_j U_j(k) H_j(k) + V_j(k) conj(H_j(-k))   (six weighted channels)
//   Y(k) = U_3(k) H_3(k)                                 (mask correlation)
//   z-axis inverse FFT of Z = X + iY at k and of conj(X) + i conj(Y) at -k,
// keeping the 2nz-1 shift planes.  Loops over the batch's rotations so the
// fixed spectra tile stays in L2.
// ---------------------------------------------------------------------------
// shared memory of a zmac block with W primary columns (see ZmacCfg)
template <int P, bool HALF, int V>
constexpr size_t zmac_smem_base(int W) {
  const int NI = HALF ? SplitV<P, V>::N1 / 2 : SplitV<P, V>::N1;
  const size_t cs = 2 * W < 16 ? FourStep<P, true, V>::CS : FourStep<P, false, V>::CS;
  return ((size_t)7 * W * P + (size_t)2 * W * cs + (size_t)2 * NI * (2 * W * SplitV<P, V>::N2)) *
         sizeof(float2);
}

template <int P, bool HALF, int V>
struct ZmacCfg {
  // primary columns per block: the block's tile of the seven fixed spectra
  // (7 * W * P complex values) stays in shared memory for the whole batch;
  // 8 columns where the tile, the exchange and two input stages fit (at most
  // 227 KB per block), else 4
  static constexpr int W =
      (P <= 320 && zmac_smem_base<P, HALF, V>(8) + P * sizeof(float2) <= 232448) ? 8 : 4;
  static constexpr int NT = 2 * W * SplitV<P, V>::N2;
  // exchange rows unpadded when 16 columns fill a half-warp (natural order)
  static constexpr bool PAD = 2 * W < 16;
  using FS = FourStep<P, PAD, V>;
  static constexpr int NI = FwdIn<FS, HALF>::NI;   // staged inputs per thread and field
  // shared memory: fixed-spectra tile [7][W][P], transform exchange [2W][CS],
  // two stages of field inputs [2][NI][NT] and, where it does not cost a
  // second block per SM, the twiddle table [P] (else twiddles come from L1)
  static constexpr size_t smem_base = zmac_smem_base<P, HALF, V>(W);
  static constexpr bool fits2(size_t b) { return 2 * (b + 1024) <= 228 * 1024; }   // per-block reserve
  static constexpr bool TWS = fits2(smem_base + P * sizeof(float2)) || !fits2(smem_base);
  static constexpr size_t smem_one = smem_base + (TWS ? P * sizeof(float2) : 0);
  // a second exchange buffer, used by alternate fields, where it fits without
  // costing a block per SM: the next field's first step then need not wait
  // for this field's multiply-accumulate to finish reading
  static constexpr size_t ex_bytes = (size_t)2 * W * FS::CS * sizeof(float2);
  static constexpr int EXB =
      (smem_one + ex_bytes <= 232448 && fits2(smem_one + ex_bytes) == fits2(smem_one)) ? 2 : 1;
  static constexpr size_t smem_bytes = smem_one + (EXB - 1) * ex_bytes;
  // Registers per thread when B blocks share an SM: each of the SM's four
  // sub-partitions holds 16384 registers and the warps placed on it, at most
  // ceil(B * warps / 4) of them (allocation in multiples of 8 per thread).
  static constexpr int regs_for(int B) {
    return (16384 / (32 * ((B * ((NT + 31) / 32) + 3) / 4))) / 8 * 8;
  }
  // two blocks per SM where shared memory allows it and each thread still
  // keeps at least 128 registers
  static constexpr int MIN_BLOCKS = (fits2(smem_bytes) && regs_for(2) >= 128) ? 2 : 1;
};

template <int P, int ST, bool HALF, int V>
__global__ void __launch_bounds__(ZmacCfg<P, HALF, V>::NT, ZmacCfg<P, HALF, V>::MIN_BLOCKS)
k_zmac(const void* __restrict__ F1, const float2* __restrict__ UV, float2* __restrict__ F2,
       const float2* __restrict__ tw, Geo g, int nrot, const int* __restrict__ bounds) {
  using C = ZmacCfg<P, HALF, V>;
  using FS = typename C::FS;
  using FI = FwdIn<FS, HALF>;
  constexpr int W = C::W;
  constexpr int N1 = FS::N1, N2 = FS::N2, CS = FS::CS, H = C::NI;
  constexpr int NC = 2 * W, NT = C::NT, MI = (W * P + NT - 1) / NT;
  constexpr int TILE = W * P;                 // complex values per fixed-spectra tile
  extern __shared__ __align__(16) float2 smem[];
  float2* uvs = smem;                         // [7][W][P] fixed-spectra weights
  constexpr int EXB = C::EXB;
  float2* ex0 = smem + 7 * TILE;              // [EXB][NC][CS] transform exchange
  float2* stage = ex0 + EXB * NC * CS;        // [2][H][NT] inputs of the next two fields
                                              // (each thread uses only its own slots)
  float2* tws = stage + 2 * H * NT;           // [P] twiddles
  // a transformed column stays in the exchange slots of the four-step split:
  // X[kz] with kz = k1 + N1*k2 sits at k2*RS + k1
  auto slot = [](int kz) { return (kz / N1) * FS::RS + kz % N1; };
  const int t = threadIdx.x;
  const int kx = blockIdx.y, ky0 = blockIdx.x * W;
  const int mkx = (g.Px - kx) % g.Px;
  const bool self_mirror = (2 * kx) % g.Px == 0;
  const long long hx = g.Px / 2 + 1;
  const long long S7 = hx * g.Py * (long long)P;
  const long long plane_stride = (long long)g.Px * g.Py;

  // step-1 role: column c1 (fastest), n2
  const int c1 = t % NC, n2 = t / NC;
  const int pk1 = ky0 + (c1 < W ? c1 : c1 - W);
  const bool ok1 = pk1 < g.Py;
  const int ky1 = c1 < W ? pk1 : (g.Py - pk1) % g.Py;
  const int kx1 = c1 < W ? kx : mkx;
  const long long col_off = (long long)kx1 * g.nz * g.Py + ky1;   // F1 is [r][j][kx][z][ky]
  // step-2 role: column c2 (fastest), k1
  const bool has2 = t < NC * N1;
  const int c2 = t % NC, k1 = t / NC;

  // z = N2*n1 + n2 < nz (with nz <= P/2 only n1 < N1/2).  Field inputs are copied
  // asynchronously (cp.async) two fields ahead into this thread's own slots of
  // two stages: no registers are held meanwhile.  Slots outside the volume are
  // zero once and never copied to.  Fields run in the order (r, j), j < nfr(r).
#pragma unroll
  for (int n1 = 0; n1 < H; ++n1) {
    const int z = N2 * n1 + n2;
    if (!(ok1 && z < g.nz)) stage[n1 * NT + t] = stage[(H + n1) * NT + t] = make_float2(0.f, 0.f);
  }
  auto nfr = [&](int r) { return (r & 1) ? g.nch : g.nf; };  // an odd rotation's mask came with its partner
  int pr = 0, pj = 0;                         // next field to copy
  auto fetch = [&](float2* buf) {             // copies field (pr, pj), if any, and advances
    if (pr < nrot) {
      const char* src = Fields<ST>::field(F1, g, g.nz * plane_stride, pr, pj);
      if (ST == kStoreF32 || pj == g.nch) {
#pragma unroll
        for (int n1 = 0; n1 < H; ++n1) {
          const int z = N2 * n1 + n2;
          if (ok1 && z < g.nz)
            cp_async8(buf + n1 * NT + t, src + (col_off + (long long)z * g.Py) * 8);
        }
      } else {
#pragma unroll
        for (int n1 = 0; n1 < H; ++n1) {
          const int z = N2 * n1 + n2;
          if (ok1 && z < g.nz)
            cp_async4(buf + n1 * NT + t, src + (col_off + (long long)z * g.Py) * 4);
        }
      }
      if (++pj == nfr(pr)) { pj = 0; ++pr; }
    }
    cp_async_commit();                         // one group per call, empty or not
  };
  // this thread's staged inputs of field j from buf, once all but the most
  // recent copy group have landed
  auto take = [&](float2 (&v)[H], const float2* buf, int j) {
    if (ST == kStoreF32 || j == g.nch) {
#pragma unroll
      for (int n1 = 0; n1 < H; ++n1) v[n1] = buf[n1 * NT + t];
    } else if (ST == kStoreBF16) {
#pragma unroll
      for (int n1 = 0; n1 < H; ++n1)
        v[n1] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(buf + n1 * NT + t));
    } else {                                   // FP16: undo the field's power-of-two scale
      const float isc = 1.0f / field_scale(g.scale1, j);
#pragma unroll
      for (int n1 = 0; n1 < H; ++n1) {
        const float2 h = __half22float2(*reinterpret_cast<const __half2*>(buf + n1 * NT + t));
        v[n1] = make_float2(h.x * isc, h.y * isc);
      }
    }
  };
  // the block's fixed-spectra tile: 7 contiguous runs of W*P values (rows
  // ky0..ky0+W-1 are contiguous in [kx][ky][kz]), copied asynchronously as the
  // first copy group; rows past Py are zero
  {
    const int valid = min(W, g.Py - ky0) * P;
    for (int a = 0; a < 2 * g.nch + 1; ++a) {
      const float2* src = UV + a * S7 + ((long long)kx * g.Py + ky0) * P;
      float2* dst = uvs + a * TILE;
      for (int q = t; q < TILE / 2; q += NT) {
        if (2 * q < valid) cp_async16(dst + 2 * q, src + 2 * q);
        else reinterpret_cast<float4*>(dst)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    cp_async_commit();
  }
  fetch(stage);
  fetch(stage + H * NT);
  constexpr bool TWS = C::TWS;
  if constexpr (TWS)
    for (int q = t; q < P; q += NT) tws[q] = __ldg(&tw[q]);
  const float2* twz = TWS ? tws : tw;
  __syncthreads();                            // twiddles visible to all (the tile is
                                              // waited for with the first field)

  // Y of an odd rotation is formed with its partner's mask field and carried
  // in Yn: live only from that product to the next rotation's start
  float2 Y[MI], Yn[MI];
  int f = 0;                                  // field counter: stage f & 1
  for (int r = 0; r < nrot; ++r) {
    float2 X[MI];
#pragma unroll
    for (int m = 0; m < MI; ++m) {
      X[m] = make_float2(0.f, 0.f);
      Y[m] = (r & 1) ? Yn[m] : make_float2(0.f, 0.f);
    }
    // Eq. 7-8: the weighted channel products (separated through the mirror
    // column) and the mask product of field j, transformed in exb,
    // accumulated in registers
    auto mac = [&](int j, const float2* exb) {
      if (j < g.nch) {
        const float2* Us = uvs + (2 * j) * TILE;
        const float2* Vs = uvs + (2 * j + 1) * TILE;
#pragma unroll
        for (int m = 0; m < MI; ++m) {
          const int i = t + NT * m;
          if (i < TILE) {
            const int c = i / P, kz = i - c * P;
            const float2 h = exb[c * CS + slot(kz)];
            const float2 hm = cconj(exb[(W + c) * CS + slot(kz == 0 ? 0 : P - kz)]);
            X[m] = cadd(X[m], cadd(cmul(Us[i], h), cmul(Vs[i], hm)));
          }
        }
      } else {
        // the mask pair (M_r, M_{r+1}): M_r = (h + hm)/2, M_{r+1} = -i (h - hm)/2
        const float2* Ms = uvs + 2 * g.nch * TILE;
#pragma unroll
        for (int m = 0; m < MI; ++m) {
          const int i = t + NT * m;
          if (i < TILE) {
            const int c = i / P, kz = i - c * P;
            const float2 h = exb[c * CS + slot(kz)];
            const float2 hm = cconj(exb[(W + c) * CS + slot(kz == 0 ? 0 : P - kz)]);
            const float2 U = Ms[i];
            Y[m] = cmul(U, cscale(cadd(h, hm), 0.5f));
            const float2 d = cscale(csub(h, hm), 0.5f);
            Yn[m] = cmul(U, make_float2(d.y, -d.x));
          }
        }
      }
    };
    // step 2 of one column sequence (column cc, k1), in place: the outputs
    // X[k1 + N1*k2] go to the slots k2*RS + k1 this thread has just read, so
    // no other thread's reads are overtaken
    auto step2_at = [&](float2* exb, int cc, int kk) {
      float2 u[N2];
      FS::template step2<-1>(u, exb + cc * CS, kk);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) exb[cc * CS + k2 * FS::RS + kk] = u[k2];
    };
#pragma unroll 1
    for (int j = 0; j < nfr(r);) {
      if (EXB == 2 && j + 1 < nfr(r)) {
        // two fields at once, in the two exchanges: both first steps, one
        // barrier, both second steps spread over all threads, one barrier,
        // both products, one barrier
        float2* ex1 = ex0 + NC * CS;
        cp_async_wait_all();                   // both fields' inputs have landed
        {
          float2 v[H];
          take(v, stage + (f & 1) * H * NT, j);
          FI::template step1<-1, TWS>(v, ex0 + c1 * CS, n2, twz);
          take(v, stage + ((f + 1) & 1) * H * NT, j + 1);
          FI::template step1<-1, TWS>(v, ex1 + c1 * CS, n2, twz);
        }
        __syncthreads();                       // (also orders this thread's reads of the
                                               //  stages before the next copies into them)
        fetch(stage + (f & 1) * H * NT);       // the next two fields
        fetch(stage + ((f + 1) & 1) * H * NT);
        for (int w = t; w < 2 * NC * N1; w += NT) {
          const int q = w < NC * N1 ? w : w - NC * N1;
          step2_at(w < NC * N1 ? ex0 : ex1, q % NC, q / NC);
        }
        __syncthreads();
        mac(j, ex0);
        mac(j + 1, ex1);
        __syncthreads();
        j += 2;
        f += 2;
      } else {
        float2* buf = stage + (f & 1) * H * NT;
        cp_async_wait_one();                   // all but the most recent copy group
        float2 v[H];
        take(v, buf, j);
        FI::template step1<-1, TWS>(v, ex0 + c1 * CS, n2, twz);
        __syncthreads();                       // (also orders this thread's reads of buf
                                               //  before the next copies into it)
        fetch(buf);                            // two fields ahead
        if (has2) step2_at(ex0, c2, k1);
        __syncthreads();
        mac(j, ex0);
        __syncthreads();
        ++j;
        ++f;
      }
    }
    float2* ex = ex0;                         // the rotation's inverse
    // Z = X + iY at k, conj(X) + i conj(Y) at -k
#pragma unroll
    for (int m = 0; m < MI; ++m) {
      const int i = t + NT * m;
      if (i < TILE) {
        const int c = i / P, kz = i - c * P;
        ex[c * CS + slot(kz)] = make_float2(X[m].x - Y[m].y, X[m].y + Y[m].x);
        ex[(W + c) * CS + slot(kz == 0 ? 0 : P - kz)] = make_float2(X[m].x + Y[m].y, Y[m].x - X[m].y);
      }
    }
    __syncthreads();
    {
      float2 v[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) v[n1] = ex[c1 * CS + slot(N2 * n1 + n2)];
      __syncthreads();
      FS::template step1<1, TWS>(v, ex + c1 * CS, n2, twz);
    }
    __syncthreads();
    if (has2 && !(c2 >= W && self_mirror)) {
      const int pk2 = ky0 + (c2 < W ? c2 : c2 - W);
      if (pk2 < g.Py) {
        const int ky2 = c2 < W ? pk2 : (g.Py - pk2) % g.Py;
        const int kx2 = c2 < W ? kx : mkx;
        float2 u[N2];
        FS::template step2<1>(u, ex + c2 * CS, k1);
        float2* dst = F2 + ((long long)r * g.Px + kx2) * g.vz * g.Py + ky2;   // [r][kx][vz][ky]
        const int lo = bounds ? bounds[6 * r] : 0, hi = bounds ? bounds[6 * r + 1] : g.vz - 1;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          const int vz = shift_slot(k1 + N1 * k2, g.nz, P, lo, hi);
          if (vz >= 0) dst[(long long)vz * g.Py] = u[k2];
        }
      }
    }
    __syncthreads();
  }
}

template <int P, bool HALF, int V>
void launch_zmac_t(const void* F1, const float2* UV, float2* F2, const float2* tw, Geo g, int nrot,
                   const int* bounds, cudaStream_t st) {
  using C = ZmacCfg<P, HALF, V>;
  dim3 grid((unsigned)((g.Py + C::W - 1) / C::W), (unsigned)(g.Px / 2 + 1));
  by_store(g.store, [&](auto sf) {
    constexpr int ST = decltype(sf)::value;
    set_smem(k_zmac<P, ST, HALF, V>, C::smem_bytes);
    k_zmac<P, ST, HALF, V><<<grid, C::NT, C::smem_bytes, st>>>(F1, UV, F2, tw, g, nrot, bounds);
  });
}

}  // namespace csngf

#include "zmac_tc.cuh"

namespace csngf {

template <int P>
void launch_zmac(const void* F1, const float2* UV, float2* F2, const float2* tw, Geo g, int nrot,
                 const int* bounds, cudaStream_t st, int v) {
  by_split<P>(v, [&](auto vc) {
    constexpr int V = decltype(vc)::value;
    const bool half = 2 * g.nz <= P;
    if (g.tc && g.store != kStoreF32) {          // reduced-precision forms: tensor-core z DFT
      bool done = false;
      by_store(g.store, [&](auto sf) {
        constexpr int ST = decltype(sf)::value;
        done = half ? launch_zsplit_t<P, ST, true, V>(F1, UV, F2, tw, g, nrot, bounds, st)
                    : launch_zsplit_t<P, ST, false, V>(F1, UV, F2, tw, g, nrot, bounds, st);
      });
      if (done) return;
    }
    if (half) launch_zmac_t<P, true, V>(F1, UV, F2, tw, g, nrot, bounds, st);
    else launch_zmac_t<P, false, V>(F1, UV, F2, tw, g, nrot, bounds, st);
  });
}

// ---------------------------------------------------------------------------
// prep_z (fixed volume, once): z-axis FFT of A's packed fields, channel
// separation via the mirror column, and the weights
//   U_j = (w_a conj(A_a) - i w_b conj(A_b)) / 2,  V_j = (w_a conj(A_a) + i w_b conj(A_b)) / 2
// for the channel fields j < nch (channels a, b of the pair with their Eq. 6
// weights, or Eq. 3 weights), and conj(A_mask) last, stored for kx <= Px/2.
// ---------------------------------------------------------------------------
template <int P, int W, bool HALF>
__global__ void __launch_bounds__(2 * W * Split<P>::N2)
k_prep_z(const float2* __restrict__ F1, float2* __restrict__ UV, const float2* __restrict__ tw,
         Geo g) {
  using FS = FourStep<P>;
  using FI = FwdIn<FS, HALF>;
  constexpr int N1 = FS::N1, N2 = FS::N2, CS = FS::CS;
  constexpr int NC = 2 * W, NT = NC * N2, MI = (W * P + NT - 1) / NT;
  extern __shared__ float2 ex[];
  const int t = threadIdx.x;
  const int kx = blockIdx.y, ky0 = blockIdx.x * W;
  const int mkx = (g.Px - kx) % g.Px;
  const long long hx = g.Px / 2 + 1;
  const long long S7 = hx * g.Py * (long long)P;
  const int c1 = t % NC, n2 = t / NC;
  const int pk1 = ky0 + (c1 < W ? c1 : c1 - W);
  const bool ok1 = pk1 < g.Py;
  const int ky1 = c1 < W ? pk1 : (g.Py - pk1) % g.Py;
  const int kx1 = c1 < W ? kx : mkx;
  const bool has2 = t < NC * N1;
  const int c2 = t % NC, k1 = t / NC;
  const long long plane_stride = (long long)g.Px * g.Py;
#pragma unroll 1
  for (int j = 0; j < g.nf; ++j) {
    // Eq. 6 weights: squared (1,1), (1,2), (2,2); unsquared (Eq. 3) (1,1), (1,0)
    float wa = 1.f, wb = 1.f;
    if (g.nch == 3) { wa = j == 2 ? 2.f : 1.f; wb = j == 0 ? 1.f : 2.f; }
    else { wb = j == 0 ? 1.f : 0.f; }
    const float2* src = F1 + (long long)j * g.nz * plane_stride;   // [j][kx][z][ky]
    float2 v[FI::NI];                     // z < nz: with nz <= P/2 the upper half is zero
#pragma unroll
    for (int n1 = 0; n1 < FI::NI; ++n1) {
      const int z = N2 * n1 + n2;
      v[n1] = (ok1 && z < g.nz) ? src[((long long)kx1 * g.nz + z) * g.Py + ky1]
                                : make_float2(0.f, 0.f);
    }
    FI::template step1<-1>(v, ex + c1 * CS, n2, tw);
    __syncthreads();
    float2 u[N2];
    if (has2) FS::template step2<-1>(u, ex + c2 * CS, k1);
    __syncthreads();
    if (has2) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) ex[c2 * CS + k1 + N1 * k2] = u[k2];
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < MI; ++m) {
      const int i = t + NT * m;
      if (i < W * P) {
        const int c = i / P, kz = i - c * P;
        const int ky = ky0 + c;
        if (ky < g.Py) {
          const float2 h = ex[c * CS + kz];
          const long long o = ((long long)kx * g.Py + ky) * P + kz;
          if (j < g.nch) {
            const float2 hm = cconj(ex[(W + c) * CS + (kz == 0 ? 0 : P - kz)]);
            // A_a = (h + hm)/2, A_b = -i (h - hm)/2
            const float2 Aa = cscale(cadd(h, hm), 0.5f);
            const float2 d = cscale(csub(h, hm), 0.5f);
            const float2 Ab = make_float2(d.y, -d.x);
            const float2 ca = cscale(cconj(Aa), wa);
            const float2 cb = cscale(cconj(Ab), wb);
            const float2 icb = make_float2(-cb.y, cb.x);          // i * cb
            UV[(2 * j) * S7 + o] = cscale(csub(ca, icb), 0.5f);
            UV[(2 * j + 1) * S7 + o] = cscale(cadd(ca, icb), 0.5f);
          } else {
            UV[2 * g.nch * S7 + o] = cconj(h);
          }
        }
      }
    }
    __syncthreads();
  }
}

template <int P>
void launch_prep_z(const float2* F1, float2* UV, const float2* tw, Geo g, cudaStream_t st) {
  constexpr int W = 8, N2 = Split<P>::N2;
  const size_t smem = (size_t)2 * W * FourStep<P>::CS * sizeof(float2);
  dim3 grid((unsigned)((g.Py + W - 1) / W), (unsigned)(g.Px / 2 + 1));
  auto go = [&](auto kern) {
    set_smem(kern, smem);
    kern<<<grid, 2 * W * N2, smem, st>>>(F1, UV, tw, g);
  };
  if (2 * g.nz <= P) go(k_prep_z<P, W, true>);
  else go(k_prep_z<P, W, false>);
}

// ---------------------------------------------------------------------------
// inv_y: y-axis inverse FFT of every (vz, kx) row of F2, keeping 2ny-1 shift
// rows, transposed so kx is contiguous.  Block: W consecutive kx rows.
// ---------------------------------------------------------------------------
template <int P, int W, int V>
__global__ void __launch_bounds__(W * SplitV<P, V>::N2)
k_inv_y(const float2* __restrict__ F2, float2* __restrict__ F3, const float2* __restrict__ tw,
        Geo g, const int* __restrict__ bounds) {
  using FS = FourStep<P, true, V>;
  constexpr int N1 = FS::N1, N2 = FS::N2, CS = FS::CS;
  extern __shared__ float2 ex[];
  const int t = threadIdx.x;
  const long long plane = blockIdx.x;               // r * vz + vz_i
  const int kx0 = blockIdx.y * W;
  const int r = (int)(plane / g.vz), vzi = (int)(plane - (long long)r * g.vz);
  int lo_y = 0, hi_y = g.vy - 1;
  if (bounds) {                                      // planes outside the shift bound: nothing to do
    if (vzi < bounds[6 * r] || vzi > bounds[6 * r + 1]) return;
    lo_y = bounds[6 * r + 2];
    hi_y = bounds[6 * r + 3];
  }
  {
    const int row = t / N2, n2 = t - row * N2;
    const int kx = kx0 + row;
    float2 v[N1];
    const float2* src = F2 + (((long long)r * g.Px + kx) * g.vz + vzi) * (long long)P;   // [r][kx][vz][ky]
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1)
      v[n1] = (kx < g.Px) ? src[N2 * n1 + n2] : make_float2(0.f, 0.f);
    FS::template step1<1>(v, ex + row * CS, n2, tw);
  }
  __syncthreads();
  if (t < W * N1) {
    const int col = t % W, k1 = t / W;
    const int kx = kx0 + col;
    if (kx < g.Px) {
      float2 u[N2];
      FS::template step2<1>(u, ex + col * CS, k1);
      float2* dst = F3 + plane * (long long)g.vy * g.Px + kx;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int vy = shift_slot(k1 + N1 * k2, g.ny, P, lo_y, hi_y);
        if (vy >= 0) dst[(long long)vy * g.Px] = u[k2];
      }
    }
  }
}

template <int P>
void launch_inv_y(const float2* F2, float2* F3, const float2* tw, Geo g, int nrot, const int* bounds,
                  cudaStream_t st, int v) {
  by_split<P>(v, [&](auto vc) {
    constexpr int V = decltype(vc)::value;
    constexpr int W = 16, N2 = SplitV<P, V>::N2;
    const size_t smem = (size_t)W * FourStep<P, true, V>::CS * sizeof(float2);
    set_smem(k_inv_y<P, W, V>, smem);
    dim3 grid((unsigned)(nrot * g.vz), (unsigned)((g.Px + W - 1) / W));
    k_inv_y<P, W, V><<<grid, W * N2, smem, st>>>(F2, F3, tw, g, bounds);
  });
}

// ---------------------------------------------------------------------------
// inv_x: x-axis inverse FFT of every (vz, vy) row of F3; at each valid shift
// s = X / N (Eq. 5) where N >= the minimum overlap, and the block's argmax is
// folded into the rotation's key with one atomicMax.  Optionally writes the
// score map (-inf where invalid).  Block: ROWS consecutive vy of one plane.
// ---------------------------------------------------------------------------
template <int P, int ROWS, int V>
__global__ void __launch_bounds__((ROWS * SplitV<P, V>::N2 + 31) / 32 * 32)
k_inv_x(const float2* __restrict__ F3, const float* __restrict__ thr,
        unsigned long long* __restrict__ keys, float* __restrict__ map,
        const float2* __restrict__ tw, Geo g, const int* __restrict__ bounds) {
  using FS = FourStep<P, true, V>;
  constexpr int N1 = FS::N1, N2 = FS::N2, CS = FS::CS, NT = (ROWS * N2 + 31) / 32 * 32;
  extern __shared__ float2 ex[];
  __shared__ unsigned long long red[NT / 32];
  const int t = threadIdx.x;
  const int plane = blockIdx.y;                       // r * vz + vz_i
  const int r = plane / g.vz, vzi = plane - r * g.vz;
  const int vy0 = blockIdx.x * ROWS;
  int lo_y = 0, hi_y = g.vy - 1, lo_x = 0, hi_x = g.vx - 1;
  if (bounds) {                                      // outside the shift bound: nothing to do
    const int* b = bounds + 6 * r;
    if (vzi < b[0] || vzi > b[1] || vy0 > b[3] || vy0 + ROWS - 1 < b[2]) return;
    lo_y = b[2]; hi_y = b[3]; lo_x = b[4]; hi_x = b[5];
  }
  if (t < ROWS * N2) {
    const int lrow = t / N2, n2 = t - lrow * N2;
    const int vyi = vy0 + lrow;
    const float2* src = F3 + ((long long)plane * g.vy + vyi) * P;
    float2 v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1)
      v[n1] = (vyi < g.vy) ? src[N2 * n1 + n2] : make_float2(0.f, 0.f);
    FS::template step1<1>(v, ex + lrow * CS, n2, tw);
  }
  __syncthreads();
  unsigned long long best = 0ull;
  if (t < ROWS * N1) {
    const int lr = t / N1, k1 = t - lr * N1;
    const int vyi = vy0 + lr;
    if (vyi < g.vy && vyi >= lo_y && vyi <= hi_y) {
      float2 u[N2];
      FS::template step2<1>(u, ex + lr * CS, k1);
      const float th = thr[r];
      const unsigned row_lin = ((unsigned)vzi * (unsigned)g.vy + (unsigned)vyi) * (unsigned)g.vx;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int vxi = shift_slot(k1 + N1 * k2, g.nx, P, lo_x, hi_x);
        if (vxi >= 0) {
          const float2 zz = u[k2];
          float s = __int_as_float(0xff800000);
          if (zz.y >= th) {
            s = __fdiv_rn(zz.x, zz.y);
            const unsigned long long key = make_key(s, row_lin + (unsigned)vxi);
            best = key > best ? key : best;
          }
          if (map) map[(long long)row_lin + vxi] = s;
        }
      }
    }
  }
  // block max
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
    best = o > best ? o : best;
  }
  if ((t & 31) == 0) red[t >> 5] = best;
  __syncthreads();
  if (t == 0) {
    unsigned long long b = 0ull;
    for (int w = 0; w < NT / 32; ++w) b = red[w] > b ? red[w] : b;
    if (b) atomicMax(&keys[r], b);
  }
}

template <int P>
void launch_inv_x(const float2* F3, const float* thr, unsigned long long* keys, float* map,
                  const float2* tw, Geo g, int nrot, const int* bounds, cudaStream_t st, int v) {
  by_split<P>(v, [&](auto vc) {
    constexpr int V = decltype(vc)::value;
    constexpr int N2 = SplitV<P, V>::N2;
    constexpr int ROWS = (256 / N2) > 0 ? (256 / N2) : 1;
    const size_t smem = (size_t)ROWS * FourStep<P, true, V>::CS * sizeof(float2);
    set_smem(k_inv_x<P, ROWS, V>, smem);
    dim3 grid((unsigned)((g.vy + ROWS - 1) / ROWS), (unsigned)(nrot * g.vz));
    k_inv_x<P, ROWS, V><<<grid, (ROWS * N2 + 31) / 32 * 32, smem, st>>>(F3, thr, keys, map, tw, g, bounds);
  });
}

#define CSNGF_INSTANTIATE_PASSES(P)                                                              \
  template void launch_fwd_x<P>(const float*, const uint8_t*, void*, const float2*, Geo, int,    \
                                cudaStream_t, int);                                              \
  template void launch_fwd_y<P>(const void*, void*, const float2*, Geo, int, cudaStream_t, int); \
  template void launch_zmac<P>(const void*, const float2*, float2*, const float2*, Geo, int,      \
                               const int*, cudaStream_t, int);                                   \
  template void launch_prep_z<P>(const float2*, float2*, const float2*, Geo, cudaStream_t);      \
  template void launch_inv_y<P>(const float2*, float2*, const float2*, Geo, int, const int*,     \
                                cudaStream_t, int);                                              \
  template void launch_inv_x<P>(const float2*, const float*, unsigned long long*, float*,        \
                                const float2*, Geo, int, const int*, cudaStream_t, int);

}  // namespace csngf
