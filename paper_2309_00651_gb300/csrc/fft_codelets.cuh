// Small in-register DFT codelets and the in-place mixed-radix stage used by every pass.
//
// Convention: forward DFT X[k] = sum_j x[j] exp(-2 pi i jk/R) (DIR = -1); inverse uses
// exp(+2 pi i jk/R) (DIR = +1), unnormalised.  Radices 2, 3, 4, 5 are written out from the
// definition; 6, 8, 9, 10, 12 and 16 are composed as P x Q in registers with compile-time
// roots of unity.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

namespace hfx {

// ----------------------------------------------------------------------------------
// complex helpers
// ----------------------------------------------------------------------------------
template <typename T> struct cx_t;
template <> struct cx_t<float> { using type = float2; };
template <> struct cx_t<double> { using type = double2; };
template <typename T> using cx = typename cx_t<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// s * i * a, s = +-1 (compile time)
template <int S, typename C> __device__ __forceinline__ C mul_si(C a) {
  if constexpr (S > 0) return mk<C>(-a.y, a.x);
  else return mk<C>(a.y, -a.x);
}

// ----------------------------------------------------------------------------------
// compile-time roots of unity: cos and sin of 2 pi num / den, by octant reduction of the
// rational angle and a Taylor series on |x| <= pi/4 (terms to x^25: error << 1 ulp).
// ----------------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double taylor_sin(double x) {
  double x2 = x * x, term = x, sum = x;
  for (int k = 1; k <= 12; ++k) { term *= -x2 / double((2 * k) * (2 * k + 1)); sum += term; }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int k = 1; k <= 12; ++k) { term *= -x2 / double((2 * k - 1) * (2 * k)); sum += term; }
  return sum;
}
struct cs_pair { double c, s; };
// cos/sin(2 pi num/den) for integers den > 0.
__host__ __device__ constexpr cs_pair cossin_2pi_frac(long long num, long long den) {
  num %= den;
  if (num < 0) num += den;
  double sgn_s = 1.0;
  if (2 * num > den) { num = den - num; sgn_s = -1.0; }           // angle -> 2 pi - angle
  // now num/den in [0, 1/2]
  double sgn_c = 1.0;
  if (4 * num > den) {                                              // angle -> pi - angle
    num = den - 2 * num; den = 2 * den; sgn_c = -1.0;
  }
  // now num/den in [0, 1/4]
  bool swap = false;
  if (8 * num > den) { num = den - 4 * num; den = 4 * den; swap = true; }  // angle -> pi/2 - angle
  double x = 2.0 * kPi * double(num) / double(den);
  double c = taylor_cos(x), s = taylor_sin(x);
  if (swap) { double t = c; c = s; s = t; }
  return cs_pair{sgn_c * c, sgn_s * s};
}

// x * w_R^(E) with w_R = exp(DIR * 2 pi i / R); exact shortcuts for multiples of pi/4.
template <int R, int E, int DIR, typename C>
__device__ __forceinline__ C twiddle(C a) {
  using T = decltype(C::x);
  constexpr int e = ((E % R) + R) % R;
  if constexpr (e == 0) {
    return a;
  } else if constexpr ((8 * e) % R == 0) {
    constexpr int o = (8 * e) / R;  // octant 1..7
    if constexpr (o == 4) return mk<C>(-a.x, -a.y);
    else if constexpr (o == 2) return mul_si<DIR>(a);    // exp(DIR i pi/2) = DIR i
    else if constexpr (o == 6) return mul_si<-DIR>(a);
    else {
      constexpr T h = T(0.70710678118654752440084436210484903928);
      // exp(DIR i o pi / 4)
      constexpr T cr = (o == 1 || o == 7) ? h : -h;
      constexpr T ci = DIR * ((o == 1 || o == 3) ? h : -h);
      return mk<C>(cr * (a.x) - ci * a.y, cr * a.y + ci * a.x);
    }
  } else {
    constexpr cs_pair w = cossin_2pi_frac(e, R);
    constexpr T cr = T(w.c);
    constexpr T ci = T(DIR * w.s);
    return mk<C>(a.x * cr - a.y * ci, a.x * ci + a.y * cr);
  }
}

template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// ----------------------------------------------------------------------------------
// base codelets
// ----------------------------------------------------------------------------------
template <int R, int DIR, typename C> struct Dft;

template <int DIR, typename C> struct Dft<1, DIR, C> {
  static __device__ __forceinline__ void run(C (&)[1]) {}
};

template <int DIR, typename C> struct Dft<2, DIR, C> {
  static __device__ __forceinline__ void run(C (&x)[2]) {
    C a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

template <int DIR, typename C> struct Dft<3, DIR, C> {
  static __device__ __forceinline__ void run(C (&x)[3]) {
    using T = decltype(C::x);
    constexpr T s3 = T(0.86602540378443864676372317075293618347);  // sin(2 pi / 3)
    C t1 = cadd(x[1], x[2]);
    C d = csub(x[1], x[2]);
    C a = mk<C>(x[0].x - T(0.5) * t1.x, x[0].y - T(0.5) * t1.y);
    C b = mul_si<DIR>(cscale(d, s3));  // DIR i s3 (x1 - x2)
    x[0] = cadd(x[0], t1);
    x[1] = cadd(a, b);
    x[2] = csub(a, b);
  }
};

template <int DIR, typename C> struct Dft<4, DIR, C> {
  static __device__ __forceinline__ void run(C (&x)[4]) {
    C s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
    C s13 = cadd(x[1], x[3]), d13 = mul_si<DIR>(csub(x[1], x[3]));
    x[0] = cadd(s02, s13);
    x[2] = csub(s02, s13);
    x[1] = cadd(d02, d13);
    x[3] = csub(d02, d13);
  }
};

template <int DIR, typename C> struct Dft<5, DIR, C> {
  static __device__ __forceinline__ void run(C (&x)[5]) {
    using T = decltype(C::x);
    constexpr T c1 = T(0.30901699437494742410229341718281905886);   // cos(2 pi/5)
    constexpr T c2 = T(-0.80901699437494742410229341718281905886);  // cos(4 pi/5)
    constexpr T s1 = T(0.95105651629515357211643933337938214340);   // sin(2 pi/5)
    constexpr T s2 = T(0.58778525229247312916870595463907276860);   // sin(4 pi/5)
    C a1 = cadd(x[1], x[4]), b1 = csub(x[1], x[4]);
    C a2 = cadd(x[2], x[3]), b2 = csub(x[2], x[3]);
    C r1 = mk<C>(x[0].x + c1 * a1.x + c2 * a2.x, x[0].y + c1 * a1.y + c2 * a2.y);
    C r2 = mk<C>(x[0].x + c2 * a1.x + c1 * a2.x, x[0].y + c2 * a1.y + c1 * a2.y);
    C i1 = mul_si<DIR>(mk<C>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
    C i2 = mul_si<DIR>(mk<C>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
    x[0] = cadd(x[0], cadd(a1, a2));
    x[1] = cadd(r1, i1);
    x[4] = csub(r1, i1);
    x[2] = cadd(r2, i2);
    x[3] = csub(r2, i2);
  }
};

// R = P * Q in registers: input index j = j1 + Q j2, output k = P k1 + k2.
template <int P, int Q, int DIR, typename C>
__device__ __forceinline__ void dft_composite(C (&x)[P * Q]) {
  constexpr int R = P * Q;
  C y[R];
  static_for<0, Q>([&](auto J1) {
    constexpr int j1 = decltype(J1)::value;
    C t[P];
#pragma unroll
    for (int j2 = 0; j2 < P; ++j2) t[j2] = x[j1 + Q * j2];
    Dft<P, DIR, C>::run(t);
    static_for<0, P>([&](auto K2) {
      constexpr int k2 = decltype(K2)::value;
      y[j1 + Q * k2] = twiddle<R, j1 * k2, DIR>(t[k2]);
    });
  });
#pragma unroll
  for (int k2 = 0; k2 < P; ++k2) {
    C t[Q];
#pragma unroll
    for (int j1 = 0; j1 < Q; ++j1) t[j1] = y[j1 + Q * k2];
    Dft<Q, DIR, C>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) x[P * k1 + k2] = t[k1];
  }
}

template <int DIR, typename C> struct Dft<6, DIR, C> {
  static __device__ __forceinline__ void run(C (&x)[6]) { dft_composite<2, 3, DIR>(x); }
};
template <int DIR, typename C> struct Dft<8, DIR, C> {
  static __device__ __forceinline__ void run(C (&x)[8]) { dft_composite<2, 4, DIR>(x); }
};
template <int DIR, typename C> struct Dft<9, DIR, C> {
  static __device__ __forceinline__ void run(C (&x)[9]) { dft_composite<3, 3, DIR>(x); }
};
template <int DIR, typename C> struct Dft<10, DIR, C> {
  static __device__ __forceinline__ void run(C (&x)[10]) { dft_composite<2, 5, DIR>(x); }
};
template <int DIR, typename C> struct Dft<12, DIR, C> {
  static __device__ __forceinline__ void run(C (&x)[12]) { dft_composite<4, 3, DIR>(x); }
};
template <int DIR, typename C> struct Dft<16, DIR, C> {
  static __device__ __forceinline__ void run(C (&x)[16]) { dft_composite<4, 4, DIR>(x); }
};

}  // namespace hfx
