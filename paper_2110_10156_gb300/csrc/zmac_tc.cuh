// z pass of the reduced-precision forms with the forward z-axis DFT of the
// channel fields on the tensor cores (tcgen05, FP32 accumulation in tensor
// memory).  Included by passes.cuh; computes exactly what k_zmac computes
// (Eq. 7-8: the weighted channel products summed in the spectrum, the mask
// product, one inverse z transform of Z = X + iY), in two kernels:
//
//   k_zx_tc  the channel fields' forward transform as a dense real DFT on the
//            tensor cores and the Eq. 7-8 sum X, written to HBM;
//   k_zinv   the mask field's FP32 forward transform and Y on the CUDA
//            cores, Z = X + iY, the inverse and the bound's planes to F2.
//
// The dense DFT: for a column b(z), z < nz, of a packed complex field and
// kz in [0, P/2]
//     C[kz][z] = cos(2 pi kz z / P),  S[kz][z] = sin(2 pi kz z / P)
//     H(kz)     = (C.re b + S.im b) + i (C.im b - S.re b)
//     H(P - kz) = (C.re b - S.im b) + i (C.im b + S.re b)
// so two M = 128 products (C and S, rows kz, K = z padded to a multiple of
// 16) give every frequency of every column.  The B operand is a tile of the
// 16-bit field values as they lie in F1 ([kx][z][ky] with (re, im) pairs):
// N-major, its columns (field, primary / mirror, column, re / im), so that
// the 8 primary columns of a row are two 16-byte copies.  Tensor memory lane
// kz then holds H at kz and P - kz of a column and of its mirror column
// (-kx, -ky), which is all the multiply-accumulate of that frequency pair
// needs.  The mask field (the overlap count N) and the inverse stay on the
// FP32 CUDA-core transforms, so N(chi) keeps FP32 accuracy.
#pragma once

#include <algorithm>

#include "tc.cuh"

namespace csngf {

// the CUDA-core half's block: W primary columns (kx, ky0 .. ky0 + W - 1) and
// their mirrors, one thread per (column, n2) of the length's radix split
template <int P, int V>
struct ZinvCfg {
  static constexpr int W = 8;
  static constexpr int NC = 2 * W;
  static constexpr int N2 = SplitV<P, V>::N2;
  static constexpr int NT = NC * N2;
  using FS = FourStep<P, (2 * W < 16), V>;
};

template <int ST>
__device__ __forceinline__ void store16(unsigned char* p, float v) {
  if constexpr (ST == kStoreBF16) *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
  else *reinterpret_cast<__half*>(p) = __float2half_rn(v);
}

// ---------------------------------------------------------------------------
// k_zx_tc forms X, the Eq. 7-8 sum of the weighted channel products, for
// every column of the half spectrum kx <= P/2, in HBM; k_zinv reads it.  X
// costs one write and one read of hx * Py * Pz complex values per rotation;
// in exchange the tensor-core kernel double-buffers its operands and keeps no
// CUDA-core transform in its per-rotation chain.
// X layout: [r][kx <= P/2][ky][kz] (kz contiguous).
//
// k_zx_tc, per block: one kx, W = 8 ky columns and their mirrors, every
// rotation of the launch; the cos / sin tiles and the block's U_j, V_j stay
// in shared memory.  Rotation r + 1's MMAs run while rotation r's products
// are summed; rotation r + 2's operand is copied (cp.async) as soon as
// rotation r's MMAs are done.  16 warps, four per tensor-memory lane quarter.
// ---------------------------------------------------------------------------
template <int P>
struct ZxTcCfg {
  static constexpr int W = 8;                          // primary columns per block
  static constexpr int NT = 512;                       // 16 warps: 4 per tensor-memory lane quarter,
                                                       // each summing two primary columns
  static constexpr int HF = P / 2;
  static constexpr bool OK = HF + 1 <= 128;
  static constexpr uint32_t TMEM_COLS = 512;           // 2 buffers x (C, S) x N <= 512 columns
  static constexpr size_t bytes(int kp, int nb, int nuv) {
    return (size_t)2 * 128 * kp * 2 + (size_t)2 * nb * kp * 2 + (size_t)nuv * W * P * 8 + 64;
  }
};

template <int P, int ST>
__global__ void __launch_bounds__(ZxTcCfg<P>::NT, 1)
k_zx_tc(const void* __restrict__ F1, const float2* __restrict__ UV, float2* __restrict__ Xg,
        const float2* __restrict__ tw, Geo g, int nrot, int KP) {
  using C = ZxTcCfg<P>;
  constexpr int W = C::W, NT = C::NT, TILE = W * P, HF = C::HF;
  const int NB = g.nch * 4 * W;                    // MMA N: (field, primary/mirror, column, re/im)
  const int NUV = 2 * g.nch;                       // U_j, V_j
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* As = smem_raw;                    // [cos | sin][128][KP], K-major
  const uint32_t tileA = 128u * (uint32_t)KP * 2u;
  const uint32_t sbo = (uint32_t)KP * 16u;
  unsigned char* Bs = As + 2 * tileA;              // [2][KP][NB], N-major
  const uint32_t stageB = (uint32_t)NB * (uint32_t)KP * 2u;
  float2* uvs = reinterpret_cast<float2*>(Bs + 2 * stageB);   // [NUV][W][P]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(uvs + (size_t)NUV * TILE);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int kx = blockIdx.y, ky0 = blockIdx.x * W;
  const int mkx = (g.Px - kx) % g.Px;
  const long long hx = g.Px / 2 + 1;
  const long long S7 = hx * g.Py * (long long)P;
  const long long E = (long long)g.nz * g.Px * g.Py;

  for (uint32_t q = t; q < 2 * stageB / 16; q += NT)
    reinterpret_cast<uint4*>(Bs)[q] = make_uint4(0u, 0u, 0u, 0u);
  {
    const int valid = min(W, g.Py - ky0) * P;
    for (int a = 0; a < NUV; ++a) {
      const float2* src = UV + a * S7 + ((long long)kx * g.Py + ky0) * P;
      float2* dst = uvs + a * TILE;
      for (int q = t; q < TILE / 2; q += NT) {
        if (2 * q < valid) cp_async16(dst + 2 * q, src + 2 * q);
        else reinterpret_cast<float4*>(dst)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  for (int m = warp; m < 128; m += NT / 32)
    for (int k = lane; k < KP; k += 32) {
      float cv = 0.f, sv = 0.f;
      if (m <= HF && k < g.nz) {
        const float2 w = __ldg(&tw[(m * k) % P]);   // exp(-2 pi i m k / P)
        cv = w.x;
        sv = -w.y;
      }
      const uint32_t off = (uint32_t)(m / 8) * sbo + (uint32_t)(k / 8) * 128u + (m % 8) * 16 + (k % 8) * 2;
      store16<ST>(As + off, cv);
      store16<ST>(As + tileA + off, sv);
    }
  if (t == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::alloc(tslot, C::TMEM_COLS);

  // operand copies of one (field, z) row: two 16-byte runs of primary
  // columns, 8 mirror values of 4 bytes; thread t takes item t % 10
  constexpr int ZSTEP = NT / 10;
  const int item = t % 10, zr0 = t / 10;
  const bool prim = item < 2;
  const int cm = item - 2;
  const bool okc = t < 10 * ZSTEP && (prim ? ky0 + 4 * item < g.Py : ky0 + cm < g.Py);
  const long long srow = prim ? (long long)kx * g.nz * g.Py + ky0 + 4 * item
                              : (long long)mkx * g.nz * g.Py + (g.Py - (ky0 + cm)) % g.Py;
  const int nrow = prim ? 8 * item : 16 + 2 * cm;
  auto fetch_b = [&](int r, int s) {
    if (r < nrot && okc) {
      unsigned char* B0 = Bs + (size_t)s * stageB;
      for (int j = 0; j < g.nch; ++j) {
        const char* src = Fields<ST>::field(F1, g, E, r, j);
        const int n = j * 4 * W + nrow;
        unsigned char* dcol = B0 + (uint32_t)(n / 8) * sbo + (n % 8) * 2;
        if (prim) {
          for (int z = zr0; z < g.nz; z += ZSTEP)
            cp_async16(dcol + (z / 8) * 128 + (z % 8) * 16, src + (srow + (long long)z * g.Py) * 4);
        } else {
          for (int z = zr0; z < g.nz; z += ZSTEP)
            cp_async4(dcol + (z / 8) * 128 + (z % 8) * 16, src + (srow + (long long)z * g.Py) * 4);
        }
      }
    }
  };
  const uint32_t idesc = tc::idesc_f16(ST == kStoreBF16, 0, 1, 128, NB);
  auto issue = [&](uint32_t tmem, int s) {         // operand stage s -> tensor-memory buffer s
    tc::fence_after_sync();
    const uint32_t a0 = tc::smem_addr(As), b0 = tc::smem_addr(Bs + (size_t)s * stageB);
    const uint32_t d0 = tmem + (uint32_t)(s * 2 * NB);
    for (int q = 0; q < KP / 16; ++q) {
      const uint64_t bd = tc::desc(b0 + q * 256, 128, sbo);
      tc::mma_f16(d0, tc::desc(a0 + q * 256, 128, sbo), bd, idesc, q > 0);
      tc::mma_f16(d0 + NB, tc::desc(a0 + tileA + q * 256, 128, sbo), bd, idesc, q > 0);
    }
    tc::commit(&mbar[s]);
  };

  fetch_b(0, 0);
  cp_async_commit();
  fetch_b(1, 1);
  cp_async_commit();
  cp_async_wait_one();                             // rotation 0's operand and the weights
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  if (t == 0 && nrot > 0) issue(tmem, 0);

  bool failed = false;
  int fail_buf = 0;
  uint32_t fail_par = 0;
  const int lq = warp & 3, cg = warp >> 2;         // lane quarter, column pair
  const int kz = lq * 32 + lane;
  const bool kz_ok = kz <= HF;
  const int kzm = kz == 0 ? 0 : P - kz;
#pragma unroll 1
  for (int r = 0; r < nrot; ++r) {
    const int s = r & 1;
    // (1) rotation r's products are done; its operand stage takes rotation r + 2
    const bool ok = tc::mbar_wait(&mbar[s], (uint32_t)((r >> 1) & 1), kTcWaitNs);
    if (__syncthreads_or(!ok)) {
      failed = true;
      fail_buf = s;
      fail_par = (uint32_t)((r >> 1) & 1);
      break;
    }
    tc::fence_after_sync();
    fetch_b(r + 2, s);
    cp_async_commit();
    // (2) rotation r + 1's operand has landed: its products start (the
    // barrier also orders rotation r - 1's tensor-memory reads of that buffer)
    if (r + 1 < nrot) {
      cp_async_wait_one();
      tc::fence_async_smem();
    }
    __syncthreads();
    if (t == 0 && r + 1 < nrot) issue(tmem, (r + 1) & 1);
    // (3) Eq. 7-8: X at kz and P - kz of this thread's four primary columns
    const uint32_t trow = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(s * 2 * NB);
    float2* Xr = Xg + (((long long)r * hx + kx) * g.Py + ky0) * P;
    {
      const int ch = cg;                           // primary columns 2 ch, 2 ch + 1
      uint32_t rc[3][4], rs[3][4], rcm[3][4], rsm[3][4];
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (j < g.nch) {
          const uint32_t col = (uint32_t)(j * 4 * W + 4 * ch);
          tc::ld4(trow + col, rc[j]);
          tc::ld4(trow + NB + col, rs[j]);
          tc::ld4(trow + 16 + col, rcm[j]);
          tc::ld4(trow + NB + 16 + col, rsm[j]);
        }
      tc::wait_ld();
      if (kz_ok) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int c = 2 * ch + i;
          if (ky0 + c >= g.Py) continue;
          float2 Xa = make_float2(0.f, 0.f), Xb = make_float2(0.f, 0.f);
#pragma unroll
          for (int j = 0; j < 3; ++j)
            if (j < g.nch) {
              const float isc = ST == kStoreF16 ? 1.0f / field_scale(g.scale1, j) : 1.0f;
              const float Cr = __uint_as_float(rc[j][2 * i]) * isc, Ci = __uint_as_float(rc[j][2 * i + 1]) * isc;
              const float Cmr = __uint_as_float(rcm[j][2 * i]) * isc;
              const float Cmi = __uint_as_float(rcm[j][2 * i + 1]) * isc;
              const float Sr = __uint_as_float(rs[j][2 * i]) * isc, Si = __uint_as_float(rs[j][2 * i + 1]) * isc;
              const float Smr = __uint_as_float(rsm[j][2 * i]) * isc;
              const float Smi = __uint_as_float(rsm[j][2 * i + 1]) * isc;
              const float2 Hk = make_float2(Cr + Si, Ci - Sr);
              const float2 Hp = make_float2(Cr - Si, Ci + Sr);
              const float2 Mk = make_float2(Cmr + Smi, Cmi - Smr);
              const float2 Mp = make_float2(Cmr - Smi, Cmi + Smr);
              const float2* Uj = uvs + (2 * j) * TILE + c * P;
              const float2* Vj = uvs + (2 * j + 1) * TILE + c * P;
              Xa = cadd(Xa, cadd(cmul(Uj[kz], Hk), cmul(Vj[kz], cconj(Mp))));
              Xb = cadd(Xb, cadd(cmul(Uj[kzm], Hp), cmul(Vj[kzm], cconj(Mk))));
            }
          Xr[c * P + kz] = Xa;
          if (kzm != kz) Xr[c * P + kzm] = Xb;
        }
      }
    }
    tc::fence_before_sync();
  }
  cp_async_wait_all();
  if (failed) {
    if (t == 0 && g.tc_err) atomicExch(g.tc_err, 1);
    tc::mbar_wait(&mbar[fail_buf], fail_par, kTcWaitNs / 4);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, C::TMEM_COLS);
}

// the CUDA-core half: mask field forward z transform, Y = conj(M_A^) M_B^,
// Z = X + iY with X from k_zx_tc, the inverse z transform and the bound's
// shift planes to F2 (the same arithmetic as k_zmac for these steps)
// Two blocks per SM (at most 96 registers a thread at the 320-thread 10 x 20
// split; a few bytes spill): its 40 KB of shared memory allow it, and the
// extra warps hide the transforms' latency (BF16 z pass 127 -> 114 ms per
// 1000 rotations of the 150^3 workload).
template <int P, int ST, bool HALF, int V>
__global__ void __launch_bounds__(ZinvCfg<P, V>::NT, 2)
k_zinv(const void* __restrict__ F1, const float2* __restrict__ Xg, const float2* __restrict__ UV,
       float2* __restrict__ F2, const float2* __restrict__ tw, Geo g, int nrot,
       const int* __restrict__ bounds) {
  using C = ZinvCfg<P, V>;
  using FS = typename C::FS;
  using FI = FwdIn<FS, HALF>;
  constexpr int W = C::W, NC = C::NC, N1 = FS::N1, N2 = FS::N2, CS = FS::CS, NT = C::NT;
  constexpr int HI = FI::NI;
  constexpr int TILE = W * P, MI = (TILE + NT - 1) / NT;
  extern __shared__ __align__(16) float2 smz[];
  float2* ex = smz;                                // [NC][CS]
  float2* Ms = ex + NC * CS;                       // [W][P] the mask weights conj(M_A^)
  float2* tws = Ms + TILE;                         // [P]
  const int t = threadIdx.x;
  const int kx = blockIdx.y, ky0 = blockIdx.x * W;
  const int mkx = (g.Px - kx) % g.Px;
  const bool self_mirror = (2 * kx) % g.Px == 0;
  const long long hx = g.Px / 2 + 1;
  const long long S7 = hx * g.Py * (long long)P;
  const long long E = (long long)g.nz * g.Px * g.Py;
  auto slot = [](int kz) { return (kz / N1) * FS::RS + kz % N1; };
  const int c1 = t % NC, n2 = t / NC;
  const int pk1 = ky0 + (c1 < W ? c1 : c1 - W);
  const bool ok1 = pk1 < g.Py;
  const int ky1 = c1 < W ? pk1 : (g.Py - pk1) % g.Py;
  const int kx1 = c1 < W ? kx : mkx;
  const long long col_off = (long long)kx1 * g.nz * g.Py + ky1;
  const bool has2 = t < NC * N1;
  const int c2 = t % NC, k1 = t / NC;

  {
    const int valid = min(W, g.Py - ky0) * P;
    const float2* src = UV + 2 * g.nch * S7 + ((long long)kx * g.Py + ky0) * P;
    for (int q = t; q < TILE / 2; q += NT) {
      if (2 * q < valid) cp_async16(Ms + 2 * q, src + 2 * q);
      else reinterpret_cast<float4*>(Ms)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    cp_async_commit();
  }
  for (int q = t; q < P; q += NT) tws[q] = __ldg(&tw[q]);
  float2 mv[HI];
  auto load_m = [&](int r) {
#pragma unroll
    for (int n1 = 0; n1 < HI; ++n1) {
      const int z = N2 * n1 + n2;
      mv[n1] = make_float2(0.f, 0.f);
      if (r < nrot && ok1 && z < g.nz) {
        const float2* src = reinterpret_cast<const float2*>(Fields<ST>::field(F1, g, E, r, g.nch));
        mv[n1] = __ldg(&src[col_off + (long long)z * g.Py]);
      }
    }
  };
  // X of this thread's (column, kz) elements, one rotation ahead
  float2 xv[MI];
  auto load_x = [&](int r) {
#pragma unroll
    for (int m = 0; m < MI; ++m) {
      const int i = t + NT * m;
      xv[m] = make_float2(0.f, 0.f);
      if (r < nrot && i < TILE) {
        const int c = i / P, kz = i - c * P;
        if (ky0 + c < g.Py) xv[m] = __ldg(&Xg[(((long long)r * hx + kx) * g.Py + ky0 + c) * P + kz]);
      }
    }
  };
  auto step2_at = [&](int cc, int kk) {
    float2 u[N2];
    FS::template step2<-1>(u, ex + cc * CS, kk);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) ex[cc * CS + k2 * FS::RS + kk] = u[k2];
  };
  load_m(0);
  load_x(0);
  cp_async_wait_all();
  __syncthreads();

  float2 Y[MI], Yn[MI];
#pragma unroll 1
  for (int r = 0; r < nrot; ++r) {
    if (!(r & 1)) {
      FI::template step1<-1, true>(mv, ex + c1 * CS, n2, tws);
      load_m(r + 2);
      __syncthreads();
      if (has2) step2_at(c2, k1);
      __syncthreads();
#pragma unroll
      for (int m = 0; m < MI; ++m) {
        const int i = t + NT * m;
        if (i < TILE) {
          const int c = i / P, kz = i - c * P;
          const float2 h = ex[c * CS + slot(kz)];
          const float2 hm = cconj(ex[(W + c) * CS + slot(kz == 0 ? 0 : P - kz)]);
          const float2 U = Ms[i];
          Y[m] = cmul(U, cscale(cadd(h, hm), 0.5f));
          const float2 d = cscale(csub(h, hm), 0.5f);
          Yn[m] = cmul(U, make_float2(d.y, -d.x));
        }
      }
      __syncthreads();
    } else {
#pragma unroll
      for (int m = 0; m < MI; ++m) Y[m] = Yn[m];
    }
    // Z = X + iY at k, conj(X) + i conj(Y) at -k
#pragma unroll
    for (int m = 0; m < MI; ++m) {
      const int i = t + NT * m;
      if (i < TILE) {
        const int c = i / P, kz = i - c * P;
        const float2 X = xv[m];
        ex[c * CS + slot(kz)] = make_float2(X.x - Y[m].y, X.y + Y[m].x);
        ex[(W + c) * CS + slot(kz == 0 ? 0 : P - kz)] = make_float2(X.x + Y[m].y, Y[m].x - X.y);
      }
    }
    load_x(r + 1);
    __syncthreads();
    {
      float2 v[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) v[n1] = ex[c1 * CS + slot(N2 * n1 + n2)];
      __syncthreads();
      FS::template step1<1, true>(v, ex + c1 * CS, n2, tws);
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

// the tensor-core z pass when g.zx (the X buffer) is set and the length,
// precision form and shared memory allow it; false otherwise (the caller then
// runs k_zmac)
template <int P, int ST, bool HALF, int V>
bool launch_zsplit_t(const void* F1, const float2* UV, float2* F2, const float2* tw, Geo g, int nrot,
                     const int* bounds, cudaStream_t st) {
  using C1 = ZxTcCfg<P>;
  using C2 = ZinvCfg<P, V>;
  if constexpr (!C1::OK || ST == kStoreF32) {
    return false;
  } else {
    if (!g.zx) return false;
    const int KP = (g.nz + 15) / 16 * 16;
    const int NB = g.nch * 4 * C1::W;
    if (NB > 128 || NB % 16 != 0) return false;
    const size_t b1 = C1::bytes(KP, NB, 2 * g.nch);
    if (b1 > 232448) return false;
    const size_t s1 = std::max<size_t>(b1, 120 * 1024);   // one block per SM: all of its tensor memory
    set_smem(k_zx_tc<P, ST>, s1);
    dim3 grid((unsigned)((g.Py + C1::W - 1) / C1::W), (unsigned)(g.Px / 2 + 1));
    k_zx_tc<P, ST><<<grid, C1::NT, s1, st>>>(F1, UV, g.zx, tw, g, nrot, KP);
    const size_t s2 = ((size_t)C2::NC * C2::FS::CS + (size_t)C2::W * P + P) * sizeof(float2);
    set_smem(k_zinv<P, ST, HALF, V>, s2);
    k_zinv<P, ST, HALF, V><<<grid, C2::NT, s2, st>>>(F1, g.zx, UV, F2, tw, g, nrot, bounds);
    return true;
  }
}

}  // namespace csngf
