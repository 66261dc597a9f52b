// z pass of the reduced-precision forms with the forward z-axis DFT of the
// channel fields on the tensor cores (tcgen05, FP32 accumulation in tensor
// memory).  Included by passes.cuh; computes exactly what k_zmac computes
// (Eq. 7-8: the weighted channel products summed in the spectrum, the mask
// product, one inverse z transform of Z = X + iY), with the channel fields'
// forward transform done as a dense real DFT:
//
//   for a column b(z), z < nz, of a packed complex field and kz in [0, P/2]
//     C[kz][z] = cos(2 pi kz z / P),  S[kz][z] = sin(2 pi kz z / P)
//     H(kz)     = (C.re b + S.im b) + i (C.im b - S.re b)
//     H(P - kz) = (C.re b - S.im b) + i (C.im b + S.re b)
//
// so two M = 128 products (C and S, rows kz, K = z padded to a multiple of
// 16) give every frequency of every column.  The B operand is a tile of the
// 16-bit field values as they lie in F1 ([kx][z][ky] with (re, im) pairs):
// N-major, its columns (field, primary / mirror, column, re / im), so that
// the 8 primary columns of a row are two 16-byte copies.  Tensor
// memory lane kz then holds H at kz and P - kz of a column and of its mirror
// column (-kx, -ky), which is all the multiply-accumulate of that frequency
// pair needs.  The mask field (the overlap count N) and the inverse keep the
// FP32 CUDA-core transforms of k_zmac, so N(chi) keeps FP32 accuracy.
//
// Per block: one kx, W = 8 ky columns and their mirrors, every rotation of
// the launch.  The block's tile of the fixed spectra stays in shared memory.
// Rotation r + 1's channel fields are multiplied while rotation r is inverse
// transformed, and as soon as those MMAs are done rotation r + 2's fields are
// copied (cp.async) into the operand, landing while rotation r + 1's mask
// field is transformed and its products summed.
#pragma once

#include <algorithm>

#include "tc.cuh"

namespace csngf {

template <int P, int V>
struct ZmacTcCfg {
  static constexpr int W = 8;                          // primary columns per block
  static constexpr int NC = 2 * W;                     // with their mirror columns
  static constexpr int N2 = SplitV<P, V>::N2;
  static constexpr int NT = NC * N2;                   // threads (the CUDA-core transforms' layout)
  static constexpr int NWF = NT / 32;                  // full warps
  static constexpr int HF = P / 2;                     // frequencies kz = 0..HF are tensor-memory lanes
  // the MAC reads tensor memory with 4 or 8 full warps (a warp reaches the
  // 32 lanes of its quarter, warp % 4)
  static constexpr bool OK = (HF + 1 <= 128) && NWF >= 4;
  static constexpr int Q = NWF >= 8 ? 2 : 1;           // warps per lane quarter
  using FS = FourStep<P, (2 * W < 16), V>;
  static constexpr uint32_t TMEM_COLS = 512;           // 2 buffers x (C, S) x N <= 512 columns
  // shared-memory bytes for K = kp (z padded to 16), N = nb, nuv fixed-spectra arrays
  static constexpr size_t bytes(int kp, int nb, int nuv) {
    return (size_t)2 * 128 * kp * 2                        // cos / sin tiles
           + (size_t)nb * kp * 2                           // channel-field operand
           + (size_t)NC * FS::CS * 8                       // transform exchange
           + (size_t)nuv * W * P * 8                       // fixed-spectra tile (U_j, V_j, mask)
           + (size_t)P * 8                                 // twiddles
           + 64;                                           // mbarriers, tensor-memory address
  }
};

template <int ST>
__device__ __forceinline__ void store16(unsigned char* p, float v) {
  if constexpr (ST == kStoreBF16) *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
  else *reinterpret_cast<__half*>(p) = __float2half_rn(v);
}

// wait limit of the tensor-core pass for its own MMAs (they take microseconds)
constexpr unsigned long long kTcWaitNs = 2000000000ull;

template <int P, int ST, bool HALF, int V>
__global__ void __launch_bounds__(ZmacTcCfg<P, V>::NT, 1)
k_zmac_tc(const void* __restrict__ F1, const float2* __restrict__ UV, float2* __restrict__ F2,
          const float2* __restrict__ tw, Geo g, int nrot, const int* __restrict__ bounds, int KP) {
  using C = ZmacTcCfg<P, V>;
  using FS = typename C::FS;
  using FI = FwdIn<FS, HALF>;
  constexpr int W = C::W, NC = C::NC, N1 = FS::N1, N2 = FS::N2, CS = FS::CS, NT = C::NT;
  constexpr int HI = FI::NI;                       // mask-field inputs per thread
  constexpr int TILE = W * P, MI = (TILE + NT - 1) / NT;
  constexpr int HF = C::HF;
  const int NB = g.nch * 4 * W;                    // MMA N: (field, column, primary/mirror, re/im)
  const int NUV = 2 * g.nch + 1;                   // U_j, V_j and the mask's weight
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* As = smem_raw;                    // [cos | sin][128][KP], K-major
  const uint32_t tileA = 128u * (uint32_t)KP * 2u;
  const uint32_t sbo = (uint32_t)KP * 16u;          // bytes between 8-row (8-column) groups
  unsigned char* Bs = As + 2 * tileA;              // [KP][NB], N-major
  const uint32_t stageB = (uint32_t)NB * (uint32_t)KP * 2u;
  float2* ex = reinterpret_cast<float2*>(Bs + stageB);   // [NC][CS]
  float2* uvs = ex + NC * CS;                      // [NUV][W][P] the block's fixed-spectra weights
  float2* tws = uvs + (size_t)NUV * TILE;          // [P] twiddles
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tws + P);   // [2] MMA completion
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int kx = blockIdx.y, ky0 = blockIdx.x * W;
  const int mkx = (g.Px - kx) % g.Px;
  const bool self_mirror = (2 * kx) % g.Px == 0;
  const long long hx = g.Px / 2 + 1;
  const long long S7 = hx * g.Py * (long long)P;
  const long long E = (long long)g.nz * g.Px * g.Py;   // complex values per F1 field
  auto slot = [](int kz) { return (kz / N1) * FS::RS + kz % N1; };

  // CUDA-core roles (the mask field's forward transform and the inverse), as in k_zmac
  const int c1 = t % NC, n2 = t / NC;
  const int pk1 = ky0 + (c1 < W ? c1 : c1 - W);
  const bool ok1 = pk1 < g.Py;
  const int ky1 = c1 < W ? pk1 : (g.Py - pk1) % g.Py;
  const int kx1 = c1 < W ? kx : mkx;
  const long long col_off = (long long)kx1 * g.nz * g.Py + ky1;
  const bool has2 = t < NC * N1;
  const int c2 = t % NC, k1 = t / NC;

  // ---------------------------------------------------------------- set-up
  for (uint32_t q = t; q < stageB / 16; q += NT)
    reinterpret_cast<uint4*>(Bs)[q] = make_uint4(0u, 0u, 0u, 0u);   // padding rows / columns stay 0
  {
    // the fixed-spectra tile: NUV runs of W*P values (rows ky0.. are contiguous
    // in [kx][ky][kz]), rows past Py zero
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
  if (warp < C::NWF) {                              // the cos and sin tiles (full warps)
    for (int m = warp; m < 128; m += C::NWF)
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
  }
  for (int q = t; q < P; q += NT) tws[q] = __ldg(&tw[q]);
  if (t == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::alloc(tslot, C::TMEM_COLS);

  // operand copies of one (field, z) row: the 8 primary columns as two
  // 16-byte runs (ky0.. is 16-byte aligned: ky0 % 8 == 0 and Py % 4 == 0) and
  // the 8 mirror columns one 4-byte value each.  Thread t takes item t % 10
  // of rows t / 10, t / 10 + NT / 10, ...
  constexpr int ZSTEP = NT / 10;
  const int item = t % 10, zr0 = t / 10;
  const bool copier = t < 10 * ZSTEP;
  const bool prim = item < 2;
  const int cm = item - 2;                         // mirror column (items 2..9)
  const bool okc = copier && (prim ? ky0 + 4 * item < g.Py : ky0 + cm < g.Py);
  const long long srow = prim ? (long long)kx * g.nz * g.Py + ky0 + 4 * item
                              : (long long)mkx * g.nz * g.Py + (g.Py - (ky0 + cm)) % g.Py;
  const int nrow = prim ? 8 * item : 16 + 2 * cm;  // N index within a field
  auto fetch_b = [&](int r) {                      // channel fields of rotation r -> the operand
    if (r < nrot && okc) {
      for (int j = 0; j < g.nch; ++j) {
        const char* src = Fields<ST>::field(F1, g, E, r, j);
        const int n = j * 4 * W + nrow;
        unsigned char* dcol = Bs + (uint32_t)(n / 8) * sbo + (n % 8) * 2;
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
  // the (FP32) mask field of an even rotation r, into registers
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

  const uint32_t idesc = tc::idesc_f16(ST == kStoreBF16, 0, 1, 128, NB);
  auto issue = [&](uint32_t tmem, int buf) {       // one thread: the operand -> buffer buf
    tc::fence_after_sync();
    const uint32_t a0 = tc::smem_addr(As), b0 = tc::smem_addr(Bs);
    const uint32_t d0 = tmem + (uint32_t)(buf * 2 * NB);
    for (int q = 0; q < KP / 16; ++q) {
      const uint64_t bd = tc::desc(b0 + q * 256, 128, sbo);
      tc::mma_f16(d0, tc::desc(a0 + q * 256, 128, sbo), bd, idesc, q > 0);
      tc::mma_f16(d0 + NB, tc::desc(a0 + tileA + q * 256, 128, sbo), bd, idesc, q > 0);
    }
    tc::commit(&mbar[buf]);
  };
  // step 2 of one column sequence, in place (as in k_zmac)
  auto step2_at = [&](int cc, int kk) {
    float2 u[N2];
    FS::template step2<-1>(u, ex + cc * CS, kk);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) ex[cc * CS + k2 * FS::RS + kk] = u[k2];
  };

  fetch_b(0);
  cp_async_commit();
  load_m(0);
  cp_async_wait_all();                             // rotation 0's operand and the weights
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  if (t == 0 && nrot > 0) issue(tmem, 0);

  float2 Y[MI], Yn[MI];
  bool failed = false;
  int fail_buf = 0;
  uint32_t fail_par = 0;
  // rotation 0's products done: the operand is free for rotation 1
  if (nrot > 0) {
    const bool ok = tc::mbar_wait(&mbar[0], 0u, kTcWaitNs);
    if (__syncthreads_or(!ok)) {
      failed = true;
      nrot = 0;                                    // skip the loop; the flag reports it
    } else {
      tc::fence_after_sync();
      fetch_b(1);
      cp_async_commit();
    }
  }
#pragma unroll 1
  for (int r = 0; r < nrot; ++r) {
    const int buf = r & 1;
    // (a) the mask field of an even rotation (its partner's mask rides in the
    // imaginary part): FP32 forward z transform, Y of this rotation and Yn of
    // the next, as in k_zmac
    if (!(r & 1)) {
      FI::template step1<-1, true>(mv, ex + c1 * CS, n2, tws);
      load_m(r + 2);                               // two rotations ahead, in flight meanwhile
      __syncthreads();
      if (has2) step2_at(c2, k1);
      __syncthreads();
      const float2* Ms = uvs + 2 * g.nch * TILE;
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
      __syncthreads();                             // the exchange is read before (d) writes it
    } else {
#pragma unroll
      for (int m = 0; m < MI; ++m) Y[m] = Yn[m];
    }
    // (d) Eq. 7-8 for the channel fields: X at kz and P - kz for this lane's
    // frequency, two primary columns at a time, from the C and S products;
    // X goes to the column's exchange slots and conj X to its mirror's
    tc::fence_after_sync();                        // the products were waited for before a barrier
    if (warp < 4 * C::Q) {
      const int lq = warp & 3, cg = warp >> 2;
      const int kz = lq * 32 + lane;
      const bool kz_ok = kz <= HF;
      const int kzm = kz == 0 ? 0 : P - kz;
      const uint32_t trow = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(buf * 2 * NB);
#pragma unroll 1
      for (int ch = cg; ch < 4; ch += C::Q) {      // two primary columns per step
        uint32_t rc[3][4], rs[3][4], rcm[3][4], rsm[3][4];   // C, S of the columns; of their mirrors
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
                const float2 Hk = make_float2(Cr + Si, Ci - Sr);       // column at kz
                const float2 Hp = make_float2(Cr - Si, Ci + Sr);       // column at P - kz
                const float2 Mk = make_float2(Cmr + Smi, Cmi - Smr);   // mirror column at kz
                const float2 Mp = make_float2(Cmr - Smi, Cmi + Smr);   // mirror column at P - kz
                const float2* Uj = uvs + (2 * j) * TILE + c * P;
                const float2* Vj = uvs + (2 * j + 1) * TILE + c * P;
                Xa = cadd(Xa, cadd(cmul(Uj[kz], Hk), cmul(Vj[kz], cconj(Mp))));
                Xb = cadd(Xb, cadd(cmul(Uj[kzm], Hp), cmul(Vj[kzm], cconj(Mk))));
              }
            ex[c * CS + slot(kz)] = Xa;
            ex[(W + c) * CS + slot(kzm)] = cconj(Xa);
            if (kzm != kz) {
              ex[c * CS + slot(kzm)] = Xb;
              ex[(W + c) * CS + slot(kz)] = cconj(Xb);
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    // (e) the next rotation's operand has landed
    if (r + 1 < nrot) {
      cp_async_wait_all();
      tc::fence_async_smem();
    }
    __syncthreads();
    // (f) its products start while this rotation's inverse runs
    if (t == 0 && r + 1 < nrot) issue(tmem, (r + 1) & 1);
    // (g) Z = X + iY at k, conj(X) + i conj(Y) at -k (X and conj X are in
    // place); inverse z transform of the 2W columns; the bound's shift planes
    // to F2 (as in k_zmac)
#pragma unroll
    for (int m = 0; m < MI; ++m) {
      const int i = t + NT * m;
      if (i < TILE) {
        const int c = i / P, kz = i - c * P;
        float2* a = ex + c * CS + slot(kz);
        float2* b = ex + (W + c) * CS + slot(kz == 0 ? 0 : P - kz);
        const float2 xa = *a, xb = *b;
        *a = make_float2(xa.x - Y[m].y, xa.y + Y[m].x);
        *b = make_float2(xb.x + Y[m].y, xb.y + Y[m].x);
      }
    }
    __syncthreads();
    {
      float2 v[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) v[n1] = ex[c1 * CS + slot(N2 * n1 + n2)];
      __syncthreads();
      FS::template step1<1, true>(v, ex + c1 * CS, n2, tws);
    }
    // rotation r + 1's products are done (by now, normally): the operand is
    // free for rotation r + 2.  The vote doubles as the step-1 barrier.
    {
      const bool ok = r + 1 < nrot ? tc::mbar_wait(&mbar[(r + 1) & 1], (uint32_t)(((r + 1) >> 1) & 1), kTcWaitNs)
                                   : true;
      if (__syncthreads_or(!ok)) {
        failed = true;
        fail_buf = (r + 1) & 1;
        fail_par = (uint32_t)(((r + 1) >> 1) & 1);
        break;
      }
      if (r + 2 < nrot) {
        tc::fence_after_sync();
        fetch_b(r + 2);
        cp_async_commit();
      }
    }
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
  cp_async_wait_all();
  if (failed) {
    if (t == 0 && g.tc_err) atomicExch(g.tc_err, 1);
    // give the MMAs still in flight a second bounded wait before their memory goes
    tc::mbar_wait(&mbar[fail_buf], fail_par, kTcWaitNs / 4);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, C::TMEM_COLS);
}

// launches k_zmac_tc when the length, the precision form and shared memory
// allow it; false otherwise (the caller then runs k_zmac)
template <int P, int ST, bool HALF, int V>
bool launch_zmac_tc_t(const void* F1, const float2* UV, float2* F2, const float2* tw, Geo g, int nrot,
                      const int* bounds, cudaStream_t st) {
  using C = ZmacTcCfg<P, V>;
  if constexpr (!C::OK || ST == kStoreF32) {
    return false;
  } else {
    const int KP = (g.nz + 15) / 16 * 16;
    const int NB = g.nch * 4 * C::W;
    if (NB > 128 || NB % 16 != 0) return false;
    const size_t bytes = C::bytes(KP, NB, 2 * g.nch + 1);
    if (bytes > 232448) return false;
    // at least 120 KB, so that one block holds an SM and all of its tensor memory
    const size_t smem = std::max<size_t>(bytes, 120 * 1024);
    set_smem(k_zmac_tc<P, ST, HALF, V>, smem);
    dim3 grid((unsigned)((g.Py + C::W - 1) / C::W), (unsigned)(g.Px / 2 + 1));
    k_zmac_tc<P, ST, HALF, V><<<grid, C::NT, smem, st>>>(F1, UV, F2, tw, g, nrot, bounds, KP);
    return true;
  }
}

}  // namespace csngf
