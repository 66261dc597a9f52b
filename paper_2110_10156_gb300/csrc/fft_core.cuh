// Register-level DFTs and the two-level (four-step) block FFT used by every
// transform pass of the all-shift NGF correlation (Eq. 7-8: the channel and
// mask correlations are evaluated in the frequency domain).
//
// Conventions: forward transforms use S = -1, X[k] = sum_n x[n] exp(-2 pi i nk/N);
// inverse transforms use S = +1 and are unnormalised.
//
// A length N = N1 * N2 transform is split as n = N2*n1 + n2, k = k1 + N1*k2:
//   step 1: for each n2, an N1-point DFT over n1 in registers, then the
//           twiddle exp(S 2 pi i n2 k1 / N), then a store to shared memory;
//   step 2: for each k1, an N2-point DFT over n2 in registers; its k2-th
//           output is X[k1 + N1*k2].
// One shared-memory exchange per transform; the caller decides where the
// step-1 inputs come from and where the step-2 outputs go.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <utility>
#include <type_traits>

namespace csngf {

// ---------------------------------------------------------------- twiddles
// Compile-time cos/sin of 2*pi*e/R from their Maclaurin series after an exact
// quadrant reduction done in integers, so quarter-turn twiddles are exact.
namespace ctw {
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double sin_series(double a) {
  double a2 = a * a, term = a, sum = a;
  for (int k = 1; k <= 14; ++k) { term *= -a2 / ((2.0 * k) * (2.0 * k + 1.0)); sum += term; }
  return sum;
}
constexpr double cos_series(double a) {
  double a2 = a * a, term = 1.0, sum = 1.0;
  for (int k = 1; k <= 14; ++k) { term *= -a2 / ((2.0 * k - 1.0) * (2.0 * k)); sum += term; }
  return sum;
}
// angle = 2*pi*e/R = q*(pi/2) + (pi/2)*rem/R with rem in [0, R)
constexpr double cos2pi(long e, long R) {
  e %= R; if (e < 0) e += R;
  long q = (4 * e) / R, rem = 4 * e - q * R;
  double a = (kPi / 2.0) * (double)rem / (double)R;
  double c = cos_series(a), s = sin_series(a);
  return (q & 3) == 0 ? c : (q & 3) == 1 ? -s : (q & 3) == 2 ? -c : s;
}
constexpr double sin2pi(long e, long R) {
  e %= R; if (e < 0) e += R;
  long q = (4 * e) / R, rem = 4 * e - q * R;
  double a = (kPi / 2.0) * (double)rem / (double)R;
  double c = cos_series(a), s = sin_series(a);
  return (q & 3) == 0 ? s : (q & 3) == 1 ? c : (q & 3) == 2 ? -s : -c;
}
}  // namespace ctw

// ---------------------------------------------------------------- complex
// Complex add and subtract as one paired FP32 instruction (add/sub.rn.f32x2:
// each lane rounds exactly as a scalar add), half the issue slots of two adds.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "add.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// asynchronous global -> shared copies (cp.async, L1-allocating); the copies a
// thread issued are visible to that thread after cp_async_wait_all()
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {   // L2 only
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (S i)
template <int S>
__device__ __forceinline__ float2 mul_si(float2 a) {
  return S < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// static for-loop with compile-time index
template <class F, int... I>
__device__ __forceinline__ void sfor_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void sfor(F&& f) {
  sfor_impl(f, std::make_integer_sequence<int, N>{});
}

// multiply by exp(S 2 pi i E / R), E a compile-time constant
template <int R, int S, int E>
__device__ __forceinline__ float2 tw_mul(float2 x) {
  constexpr int e = ((E % R) + R) % R;
  if constexpr (e == 0) {
    return x;
  } else if constexpr (2 * e == R) {
    return make_float2(-x.x, -x.y);
  } else if constexpr (4 * e == R) {
    return mul_si<S>(x);
  } else if constexpr (4 * e == 3 * R) {
    return mul_si<-S>(x);
  } else {
    constexpr float c = (float)ctw::cos2pi(e, R);
    constexpr float s = (float)(S * ctw::sin2pi(e, R));
    return make_float2(x.x * c - x.y * s, x.x * s + x.y * c);
  }
}

// ---------------------------------------------------------------- DFTs
template <int R, int S>
struct Dft;

template <int S>
struct Dft<1, S> {
  __device__ __forceinline__ static void run(float2 (&)[1]) {}
};

template <int S>
struct Dft<2, S> {
  __device__ __forceinline__ static void run(float2 (&v)[2]) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int S>
struct Dft<3, S> {
  __device__ __forceinline__ static void run(float2 (&v)[3]) {
    constexpr float c1 = (float)ctw::cos2pi(1, 3), s1 = (float)ctw::sin2pi(1, 3);
    const float2 t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const float2 x0 = v[0];
    v[0] = cadd(x0, t);
    const float2 a = make_float2(x0.x + c1 * t.x, x0.y + c1 * t.y);
    const float2 ib = mul_si<S>(make_float2(s1 * d.x, s1 * d.y));   // S i sin(2 pi/3) (x1 - x2)
    // X1 = a + S i b, X2 = a - S i b
    v[1] = cadd(a, ib);
    v[2] = csub(a, ib);
  }
};

template <int S>
struct Dft<4, S> {
  __device__ __forceinline__ static void run(float2 (&v)[4]) {
    float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    float2 b0 = cadd(v[1], v[3]), b1 = mul_si<S>(csub(v[1], v[3]));
    v[0] = cadd(a0, b0);
    v[2] = csub(a0, b0);
    v[1] = cadd(a1, b1);
    v[3] = csub(a1, b1);
  }
};

template <int S>
struct Dft<5, S> {
  __device__ __forceinline__ static void run(float2 (&v)[5]) {
    constexpr float c1 = (float)ctw::cos2pi(1, 5), c2 = (float)ctw::cos2pi(2, 5);
    constexpr float s1 = (float)ctw::sin2pi(1, 5), s2 = (float)ctw::sin2pi(2, 5);
    float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    float2 x0 = v[0];
    v[0] = cadd(x0, cadd(t1, t2));
    float2 a1 = make_float2(x0.x + c1 * t1.x + c2 * t2.x, x0.y + c1 * t1.y + c2 * t2.y);
    float2 a2 = make_float2(x0.x + c2 * t1.x + c1 * t2.x, x0.y + c2 * t1.y + c1 * t2.y);
    float2 b1 = make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
    float2 b2 = make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
    // forward: X1 = a1 - i b1, X4 = a1 + i b1, X2 = a2 - i b2, X3 = a2 + i b2
    float2 ib1 = mul_si<S>(b1), ib2 = mul_si<S>(b2);   // S i b
    v[1] = cadd(a1, ib1);
    v[4] = csub(a1, ib1);
    v[2] = cadd(a2, ib2);
    v[3] = csub(a2, ib2);
  }
};

constexpr int first_factor(int R) {
  return (R % 4 == 0 && R != 4) ? 4
         : (R % 2 == 0 && R != 2) ? 2
         : (R % 5 == 0 && R != 5) ? 5
         : (R % 3 == 0 && R != 3) ? 3
                                  : R;
}

// composite R = A * B in registers (same split as the block four-step)
template <int R, int S>
struct Dft {
  static constexpr int A = first_factor(R);
  static constexpr int B = R / A;
  static_assert(A * B == R && A > 1 && B > 1, "unsupported DFT length");
  __device__ __forceinline__ static void run(float2 (&v)[R]) {
    float2 t[B][A];
    sfor<B>([&](auto bc) {
      constexpr int b = decltype(bc)::value;
      float2 s[A];
      sfor<A>([&](auto ac) { constexpr int a = decltype(ac)::value; s[a] = v[B * a + b]; });
      Dft<A, S>::run(s);
      sfor<A>([&](auto kc) {
        constexpr int ka = decltype(kc)::value;
        t[b][ka] = tw_mul<R, S, b * ka>(s[ka]);
      });
    });
    sfor<A>([&](auto kc) {
      constexpr int ka = decltype(kc)::value;
      float2 u[B];
      sfor<B>([&](auto bc) { constexpr int b = decltype(bc)::value; u[b] = t[b][ka]; });
      Dft<B, S>::run(u);
      sfor<B>([&](auto kb) { constexpr int k = decltype(kb)::value; v[ka + A * k] = u[k]; });
    });
  }
};

// ---------------------------------------------------------------- four-step
// N = N1 * N2 with N1 <= N2 (step 2 then has at most one item per thread).
// Split variant V = 0 is the built-in choice; V = 1, where a length has one,
// is the alternative the autotuner times against it.
template <int N, int V>
struct SplitV;
template <> struct SplitV<16, 0>  { static constexpr int N1 = 4,  N2 = 4; };
template <> struct SplitV<32, 0>  { static constexpr int N1 = 4,  N2 = 8; };
template <> struct SplitV<40, 0>  { static constexpr int N1 = 4,  N2 = 10; };
template <> struct SplitV<64, 0>  { static constexpr int N1 = 8,  N2 = 8; };
template <> struct SplitV<80, 0>  { static constexpr int N1 = 8,  N2 = 10; };
template <> struct SplitV<100, 0> { static constexpr int N1 = 10, N2 = 10; };
template <> struct SplitV<128, 0> { static constexpr int N1 = 8,  N2 = 16; };
template <> struct SplitV<160, 0> { static constexpr int N1 = 8,  N2 = 20; };
template <> struct SplitV<192, 0> { static constexpr int N1 = 12, N2 = 16; };
template <> struct SplitV<200, 0> { static constexpr int N1 = 10, N2 = 20; };
template <> struct SplitV<216, 0> { static constexpr int N1 = 12, N2 = 18; };
template <> struct SplitV<256, 0> { static constexpr int N1 = 16, N2 = 16; };
template <> struct SplitV<320, 0> { static constexpr int N1 = 16, N2 = 20; };
template <> struct SplitV<360, 0> { static constexpr int N1 = 18, N2 = 20; };
template <> struct SplitV<400, 0> { static constexpr int N1 = 16, N2 = 25; };
template <> struct SplitV<512, 0> { static constexpr int N1 = 16, N2 = 32; };
template <> struct SplitV<64, 1>  { static constexpr int N1 = 4,  N2 = 16; };
template <> struct SplitV<80, 1>  { static constexpr int N1 = 4,  N2 = 20; };
template <> struct SplitV<128, 1> { static constexpr int N1 = 4,  N2 = 32; };
template <> struct SplitV<160, 1> { static constexpr int N1 = 10, N2 = 16; };
template <> struct SplitV<192, 1> { static constexpr int N1 = 8,  N2 = 24; };
template <> struct SplitV<200, 1> { static constexpr int N1 = 8,  N2 = 25; };
template <> struct SplitV<216, 1> { static constexpr int N1 = 8,  N2 = 27; };
template <> struct SplitV<256, 1> { static constexpr int N1 = 8,  N2 = 32; };
template <> struct SplitV<320, 1> { static constexpr int N1 = 10, N2 = 32; };
template <> struct SplitV<400, 1> { static constexpr int N1 = 20, N2 = 20; };
// lengths with a second split
constexpr bool has_alt_split(int N) {
  return N == 64 || N == 80 || N == 128 || N == 160 || N == 192 || N == 200 || N == 216 || N == 256 ||
         N == 320 || N == 400;
}
template <int N>
using Split = SplitV<N, 0>;

template <int N, bool PAD_ROWS = true, int V = 0>
struct FourStep {
  static constexpr int N1 = SplitV<N, V>::N1;
  static constexpr int N2 = SplitV<N, V>::N2;
  // exchange layout per sequence: [n2][k1] with padded strides (odd strides keep
  // 16 consecutive lanes on distinct bank pairs for either lane ordering).
  // Without row padding (RS = N1) a transformed sequence is in natural order;
  // that suits callers whose lanes run over sequences (the odd CS spreads them).
  static constexpr int RS = (PAD_ROWS && N1 % 2 == 0) ? N1 + 1 : N1;
  static constexpr int CS0 = N2 * RS;
  static constexpr int CS = (CS0 % 2 == 0) ? CS0 + 1 : CS0;
  static_assert(CS >= N, "sequence stride must hold N natural-order values");

  // twiddle table read: shared memory (TS) or the read-only global path
  template <bool TS>
  __device__ __forceinline__ static float2 twl(const float2* p) {
    if constexpr (TS) return *p; else return __ldg(p);
  }

  // v holds x[N2*n1 + n2] for n1 = 0..N1-1; writes twiddled N1-point outputs
  template <int S, bool TS = false>
  __device__ __forceinline__ static void step1(float2 (&v)[N1], float2* ex_seq, int n2,
                                               const float2* __restrict__ twN) {
    Dft<N1, S>::run(v);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      float2 w = twl<TS>(&twN[n2 * k1]);
      if (S > 0) w.y = -w.y;
      ex_seq[n2 * RS + k1] = (k1 == 0) ? v[k1] : cmul(v[k1], w);
    }
  }

  // Same as step1 when the input is zero for n1 >= N1/2 (a forward transform
  // of data zero-padded from length <= N/2): the N1-point DFT splits into two
  // N1/2-point DFTs, X[2m] = DFT(x)[m], X[2m+1] = DFT(x * W_N1^n)[m].
  static constexpr int H = N1 / 2;
  template <int S, bool TS = false>
  __device__ __forceinline__ static void step1_half(float2 (&v)[H], float2* ex_seq, int n2,
                                                    const float2* __restrict__ twN) {
    static_assert(N1 % 2 == 0, "half-zero step needs an even N1");
    float2 e[H], o[H];
    sfor<H>([&](auto nc) {
      constexpr int n = decltype(nc)::value;
      e[n] = v[n];
      o[n] = tw_mul<N1, S, n>(v[n]);
    });
    Dft<H, S>::run(e);
    Dft<H, S>::run(o);
#pragma unroll
    for (int m = 0; m < H; ++m) {
      const int ke = 2 * m, ko = 2 * m + 1;
      float2 we = twl<TS>(&twN[n2 * ke]), wo = twl<TS>(&twN[n2 * ko]);
      if (S > 0) { we.y = -we.y; wo.y = -wo.y; }
      ex_seq[n2 * RS + ke] = (m == 0) ? e[m] : cmul(e[m], we);
      ex_seq[n2 * RS + ko] = cmul(o[m], wo);
    }
  }

  // u[k2] = X[k1 + N1*k2]
  template <int S>
  __device__ __forceinline__ static void step2(float2 (&u)[N2], const float2* ex_seq, int k1) {
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) u[n2] = ex_seq[n2 * RS + k1];
    Dft<N2, S>::run(u);
  }
};

}  // namespace csngf
