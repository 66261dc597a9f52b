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
// N-major, its columns (field, column, primary / mirror, re / im).  Tensor
// memory lane kz then holds H at kz and P - kz of a column and of its mirror
// column (-kx, -ky), which is all the multiply-accumulate of that frequency
// pair needs.  The mask field (the overlap count N) and the inverse keep the
// FP32 CUDA-core transforms of k_zmac, so N(chi) keeps FP32 accuracy.
//
// Per block: one kx, W = 8 ky columns and their mirrors, every rotation of
// the launch.  The channel fields of rotation r + 1 are copied (cp.async) and
// multiplied while rotation r's products are summed and inverse transformed;
// the accumulators alternate between two tensor-memory buffers.
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
  // shared-memory bytes for K = kp (z padded to 16), N = nb, stages of B
  static constexpr size_t bytes(int kp, int nb, int stages, int ni) {
    return (size_t)2 * 128 * kp * 2                        // cos / sin tiles
           + (size_t)stages * nb * kp * 2                  // channel-field operand stages
           + (size_t)NC * FS::CS * 8                       // transform exchange
           + (size_t)ni * NT * 8                           // mask-field inputs
           + (size_t)W * P * 8                             // X of the primary columns
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
          const float2* __restrict__ tw, Geo g, int nrot, const int* __restrict__ bounds, int KP,
          int NSTG) {
  using C = ZmacTcCfg<P, V>;
  using FS = typename C::FS;
  using FI = FwdIn<FS, HALF>;
  constexpr int W = C::W, NC = C::NC, N1 = FS::N1, N2 = FS::N2, CS = FS::CS, NT = C::NT;
  constexpr int HI = FI::NI;                       // mask-field inputs per thread
  constexpr int TILE = W * P, MI = (TILE + NT - 1) / NT;
  constexpr int HF = C::HF;
  const int NB = g.nch * 4 * W;                    // MMA N: (field, column, primary/mirror, re/im)
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* As = smem_raw;                    // [cos | sin][128][KP], K-major
  const uint32_t tileA = 128u * (uint32_t)KP * 2u;
  const uint32_t sbo = (uint32_t)KP * 16u;          // bytes between 8-row (8-column) groups
  unsigned char* Bs = As + 2 * tileA;              // [NSTG][KP][NB], N-major
  const uint32_t stageB = (uint32_t)NB * (uint32_t)KP * 2u;
  float2* ex = reinterpret_cast<float2*>(Bs + (size_t)NSTG * stageB);   // [NC][CS]
  float2* mst = ex + NC * CS;                      // [HI][NT] mask-field inputs (own slots)
  float2* Xs = mst + HI * NT;                      // [W][P] X of the primary columns
  float2* tws = Xs + TILE;                         // [P] twiddles
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
  for (uint32_t q = t; q < (uint32_t)NSTG * stageB / 16; q += NT)
    reinterpret_cast<uint4*>(Bs)[q] = make_uint4(0u, 0u, 0u, 0u);   // padding rows / columns stay 0
  for (int q = t; q < 128 * KP; q += NT) {          // the cos and sin tiles
    const int m = q / KP, k = q - (q / KP) * KP;
    float cv = 0.f, sv = 0.f;
    if (m <= HF && k < g.nz) {
      const float2 w = __ldg(&tw[(m * k) % P]);    // exp(-2 pi i m k / P)
      cv = w.x;
      sv = -w.y;
    }
    const uint32_t off = (uint32_t)(m / 8) * sbo + (uint32_t)(k / 8) * 128u + (m % 8) * 16 + (k % 8) * 2;
    store16<ST>(As + off, cv);
    store16<ST>(As + tileA + off, sv);
  }
  for (int q = t; q < P; q += NT) tws[q] = __ldg(&tw[q]);
#pragma unroll
  for (int n1 = 0; n1 < HI; ++n1) {
    const int z = N2 * n1 + n2;
    if (!(ok1 && z < g.nz)) mst[n1 * NT + t] = make_float2(0.f, 0.f);
  }
  if (t == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::alloc(tslot, C::TMEM_COLS);

  // this thread's data column for the operand copies: primary column cq or
  // the mirror of column cq - W, N index within a field nq, z rows zq0 + N2 i
  const int cq = t % NC, zq0 = t / NC;
  const int cc_ = cq < W ? cq : cq - W;
  const int pkq = ky0 + cc_;
  const bool okq = pkq < g.Py;
  const int kyq = cq < W ? pkq : (g.Py - pkq) % g.Py;
  const int kxq = cq < W ? kx : mkx;
  const long long qoff = (long long)kxq * g.nz * g.Py + kyq;
  const int nq = 4 * cc_ + (cq < W ? 0 : 2);
  auto fetch_b = [&](int r, int s) {               // channel fields of rotation r -> stage s
    if (r < nrot && okq) {
      unsigned char* dst0 = Bs + (size_t)s * stageB;
      for (int j = 0; j < g.nch; ++j) {
        const char* src = Fields<ST>::field(F1, g, E, r, j);
        const int n = j * 4 * W + nq;
        unsigned char* dcol = dst0 + (uint32_t)(n / 8) * sbo + (n % 8) * 2;
        for (int z = zq0; z < g.nz; z += N2)
          cp_async4(dcol + (z / 8) * 128 + (z % 8) * 16, src + (qoff + (long long)z * g.Py) * 4);
      }
    }
  };
  auto fetch_m = [&](int r) {                      // the (FP32) mask field of rotation r
    if (r < nrot) {
      const char* src = Fields<ST>::field(F1, g, E, r, g.nch);
#pragma unroll
      for (int n1 = 0; n1 < HI; ++n1) {
        const int z = N2 * n1 + n2;
        if (ok1 && z < g.nz) cp_async8(mst + n1 * NT + t, src + (col_off + (long long)z * g.Py) * 8);
      }
    }
  };

  const uint32_t idesc = tc::idesc_f16(ST == kStoreBF16, 0, 1, 128, NB);
  auto issue = [&](uint32_t tmem, int s, int buf) {   // one thread: rotation in stage s -> buffer buf
    tc::fence_after_sync();
    const uint32_t a0 = tc::smem_addr(As), b0 = tc::smem_addr(Bs + (size_t)s * stageB);
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

  fetch_b(0, 0);
  fetch_m(0);
  cp_async_commit();
  if (NSTG == 2) fetch_b(1, 1);
  cp_async_commit();
  cp_async_wait_one();                             // rotation 0's operands
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  if (t == 0 && nrot > 0) issue(tmem, 0, 0);

  float2 Y[MI], Yn[MI];
  bool failed = false;
  int fail_buf = 0;
  uint32_t fail_par = 0;
#pragma unroll 1
  for (int r = 0; r < nrot; ++r) {
    const int buf = r & 1;
    // (a) the mask field of an even rotation (its partner's mask rides in the
    // imaginary part): FP32 forward z transform, Y of this rotation and Yn of
    // the next, as in k_zmac
    if (!(r & 1)) {
      float2 v[HI];
#pragma unroll
      for (int n1 = 0; n1 < HI; ++n1) v[n1] = mst[n1 * NT + t];
      FI::template step1<-1, true>(v, ex + c1 * CS, n2, tws);
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
          const int ky = ky0 + c;
          const float2 U = ky < g.Py ? __ldg(&UV[2 * g.nch * S7 + ((long long)kx * g.Py + ky) * P + kz])
                                     : make_float2(0.f, 0.f);
          Y[m] = cmul(U, cscale(cadd(h, hm), 0.5f));
          const float2 d = cscale(csub(h, hm), 0.5f);
          Yn[m] = cmul(U, make_float2(d.y, -d.x));
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < MI; ++m) Y[m] = Yn[m];
    }
    // (b) this rotation's channel spectra are in tensor-memory buffer buf
    const bool ok = tc::mbar_wait(&mbar[buf], (uint32_t)((r >> 1) & 1), kTcWaitNs);
    if (__syncthreads_or(!ok)) {
      failed = true;
      fail_buf = buf;
      fail_par = (uint32_t)((r >> 1) & 1);
      break;
    }
    tc::fence_after_sync();
    // (c) its operand stage is free: copy the channel fields NSTG rotations
    // ahead (and the next even rotation's mask field) into it
    {
      const int rn = r + NSTG;
      fetch_b(rn, NSTG == 2 ? buf : 0);
      if (!(rn & 1)) fetch_m(rn);
      cp_async_commit();
    }
    // (d) Eq. 7-8 for the channel fields: X at kz and P - kz for this lane's
    // frequency, four primary columns at a time, from the C and S products
    if (warp < 4 * C::Q) {
      const int lq = warp & 3, cg = warp >> 2;
      const int kz = lq * 32 + lane;
      const bool kz_ok = kz <= HF;
      const int kzm = kz == 0 ? 0 : P - kz;
      const uint32_t trow = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(buf * 2 * NB);
#pragma unroll 1
      for (int ch = cg; ch < 2; ch += C::Q) {
        float2 Xa[4], Xb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) Xa[i] = Xb[i] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int j = 0; j < g.nch; ++j) {
          uint32_t rc[16], rs[16];
          tc::ld16(trow + (uint32_t)(j * 4 * W + 16 * ch), rc);
          tc::ld16(trow + (uint32_t)(NB + j * 4 * W + 16 * ch), rs);
          tc::wait_ld();
          const float isc = ST == kStoreF16 ? 1.0f / field_scale(g.scale1, j) : 1.0f;
          if (kz_ok) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int ky = ky0 + 4 * ch + i;
              if (ky < g.Py) {
                const float Cr = __uint_as_float(rc[4 * i]) * isc, Ci = __uint_as_float(rc[4 * i + 1]) * isc;
                const float Cmr = __uint_as_float(rc[4 * i + 2]) * isc, Cmi = __uint_as_float(rc[4 * i + 3]) * isc;
                const float Sr = __uint_as_float(rs[4 * i]) * isc, Si = __uint_as_float(rs[4 * i + 1]) * isc;
                const float Smr = __uint_as_float(rs[4 * i + 2]) * isc, Smi = __uint_as_float(rs[4 * i + 3]) * isc;
                const float2 Hk = make_float2(Cr + Si, Ci - Sr);       // column at kz
                const float2 Hp = make_float2(Cr - Si, Ci + Sr);       // column at P - kz
                const float2 Mk = make_float2(Cmr + Smi, Cmi - Smr);   // mirror column at kz
                const float2 Mp = make_float2(Cmr - Smi, Cmi + Smr);   // mirror column at P - kz
                const long long base = ((long long)kx * g.Py + ky) * P;
                const float2* Uj = UV + (2 * j) * S7 + base;
                const float2* Vj = UV + (2 * j + 1) * S7 + base;
                Xa[i] = cadd(Xa[i], cadd(cmul(__ldg(&Uj[kz]), Hk), cmul(__ldg(&Vj[kz]), cconj(Mp))));
                Xb[i] = cadd(Xb[i], cadd(cmul(__ldg(&Uj[kzm]), Hp), cmul(__ldg(&Vj[kzm]), cconj(Mk))));
              }
            }
          }
        }
        if (kz_ok) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int c = 4 * ch + i;
            Xs[c * P + kz] = Xa[i];
            if (kzm != kz) Xs[c * P + kzm] = Xb[i];
          }
        }
      }
    }
    tc::fence_before_sync();
    // (e) the next rotation's operands have landed (all but the copies just issued)
    if (r + 1 < nrot) {
      if (NSTG == 2) cp_async_wait_one();
      else cp_async_wait_all();
      tc::fence_async_smem();
    }
    __syncthreads();
    // (f) its products start while this rotation's inverse runs
    if (t == 0 && r + 1 < nrot) issue(tmem, NSTG == 2 ? ((r + 1) & 1) : 0, (r + 1) & 1);
    // (g) Z = X + iY at k, conj(X) + i conj(Y) at -k; inverse z transform of
    // the 2W columns; the bound's shift planes to F2 (as in k_zmac)
#pragma unroll
    for (int m = 0; m < MI; ++m) {
      const int i = t + NT * m;
      if (i < TILE) {
        const int c = i / P, kz = i - c * P;
        const float2 X = Xs[i];
        ex[c * CS + slot(kz)] = make_float2(X.x - Y[m].y, X.y + Y[m].x);
        ex[(W + c) * CS + slot(kz == 0 ? 0 : P - kz)] = make_float2(X.x + Y[m].y, Y[m].x - X.y);
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
    constexpr int NI = FwdIn<typename C::FS, HALF>::NI;
    constexpr size_t kMax = 232448;
    int nstg = C::bytes(KP, NB, 2, NI) <= kMax ? 2 : (C::bytes(KP, NB, 1, NI) <= kMax ? 1 : 0);
    if (!nstg) return false;
    // at least 120 KB, so that one block holds an SM and all of its tensor memory
    const size_t smem = std::max<size_t>(C::bytes(KP, NB, nstg, NI), 120 * 1024);
    set_smem(k_zmac_tc<P, ST, HALF, V>, smem);
    dim3 grid((unsigned)((g.Py + C::W - 1) / C::W), (unsigned)(g.Px / 2 + 1));
    k_zmac_tc<P, ST, HALF, V><<<grid, C::NT, smem, st>>>(F1, UV, F2, tw, g, nrot, bounds, KP, nstg);
    return true;
  }
}

}  // namespace csngf
