// Radix-2/3/4/5/8/16/32 Stockham FFT building blocks shared by every FFT pass kernel.
//
// The FFT passes implement the FFT[...] / FFT^-1[...] of the padded PSF convolution
// (Sec. 3.3.2) and the oversampled-grid transforms of the measurement operator R (Eq. rime)
// and its adjoint. Lengths are L = c 2^k with an odd part c made of factors 3 and 5 (the
// reduced-padding PSF transforms use 3 2^k and 5 2^k; everything else is a power of two): one
// radix-3 or radix-5 stage per odd factor runs first, then the power-of-two stages.
//
// A Stockham stage with radix R and current sub-transform size Ns maps, for each butterfly
// task j in [0, L/R):
//     k = j mod Ns
//     v[r] = x[j + r L/R] * w^(r k),  w = exp(dir 2 pi i / (Ns R))
//     v    = DFT_R(v)
//     y[(j / Ns) Ns R + k + r Ns] = v[r]
// which leaves the result in natural order after the last stage (no bit reversal).
// Twiddles come from a per-length table tw[m] = exp(-2 pi i m / L) (conjugated for dir = +1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef FR_HD
#define FR_HD __host__ __device__ __forceinline__
#endif

namespace fr {

FR_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
FR_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
FR_HD float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
FR_HD float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
FR_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
FR_HD float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by dir * i  (dir = -1: -i, dir = +1: +i)
template <int DIR>
FR_HD float2 mul_i(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// ---------------------------------------------------------------------------------------
// In-register DFTs of size 2, 3, 4, 5, 8, 16, 32 with exponent sign DIR (-1 forward, +1 inverse).
// Input and output in natural order.
// ---------------------------------------------------------------------------------------
template <int DIR>
FR_HD void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <int DIR>
FR_HD void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  // X[k] = sum_n x[n] w4^(nk),  w4 = exp(DIR 2 pi i / 4) = DIR * i
  float2 s02 = cadd(x0, x2), d02 = csub(x0, x2);
  float2 s13 = cadd(x1, x3), d13 = mul_i<DIR>(csub(x1, x3));
  x0 = cadd(s02, s13);
  x2 = csub(s02, s13);
  x1 = cadd(d02, d13);
  x3 = csub(d02, d13);
}

template <int DIR>
FR_HD void dft8(float2* v) {
  const float h = 0.70710678118654752440f;
  // split into even / odd halves (decimation in time)
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  // twiddles w8^k, w8 = exp(DIR 2 pi i / 8)
  // k=1: (h, DIR h); k=2: DIR i; k=3: (-h, DIR h)
  float2 t1 = make_float2(h * (o1.x - DIR * o1.y), h * (o1.y + DIR * o1.x));
  float2 t2 = mul_i<DIR>(o2);
  float2 t3 = make_float2(-h * (o3.x + DIR * o3.y), h * (DIR * o3.x - o3.y));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1);
  v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2);
  v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3);
  v[7] = csub(e3, t3);
}

template <int DIR>
FR_HD float2 tw16(float2 a, int k) {
  // a * exp(DIR 2 pi i k / 16) for k in [0, 9], constants folded after unrolling
  const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
  const float h = 0.70710678118654752440f;
  float c, s;
  switch (k) {
    case 0: return a;
    case 1: c = c1; s = s1; break;
    case 2: c = h; s = h; break;
    case 3: c = s1; s = c1; break;
    case 4: return mul_i<DIR>(a);
    case 6: c = -h; s = h; break;
    case 9: c = -c1; s = -s1; break;
    default: c = 1.f; s = 0.f; break;
  }
  s = DIR * s;
  return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

template <int DIR>
FR_HD void dft16(float2* v) {
  // 16 = 4 x 4: n = n1 + 4 n2, k = k2 + 4 k1
  // step 1: for each n1, DFT4 over n2 -> index k2;  step 2: twiddle w16^(n1 k2);
  // step 3: for each k2, DFT4 over n1 -> k1
  float2 a[4][4];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    a[n1][0] = v[n1];
    a[n1][1] = v[n1 + 4];
    a[n1][2] = v[n1 + 8];
    a[n1][3] = v[n1 + 12];
    dft4<DIR>(a[n1][0], a[n1][1], a[n1][2], a[n1][3]);
  }
#pragma unroll
  for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
    for (int k2 = 1; k2 < 4; ++k2) a[n1][k2] = tw16<DIR>(a[n1][k2], n1 * k2);
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    float2 b0 = a[0][k2], b1 = a[1][k2], b2 = a[2][k2], b3 = a[3][k2];
    dft4<DIR>(b0, b1, b2, b3);
    v[k2] = b0;
    v[k2 + 4] = b1;
    v[k2 + 8] = b2;
    v[k2 + 12] = b3;
  }
}

// a * exp(DIR 2 pi i k / 32) for k in [0, 16): cos and sin of k pi / 16, folded after unrolling
template <int DIR>
FR_HD float2 tw32(float2 a, int k) {
  constexpr float C[16] = {1.f,
                           0.98078528040323044913f,
                           0.92387953251128675613f,
                           0.83146961230254523708f,
                           0.70710678118654752440f,
                           0.55557023301960222474f,
                           0.38268343236508977173f,
                           0.19509032201612826785f,
                           0.f,
                           -0.19509032201612826785f,
                           -0.38268343236508977173f,
                           -0.55557023301960222474f,
                           -0.70710678118654752440f,
                           -0.83146961230254523708f,
                           -0.92387953251128675613f,
                           -0.98078528040323044913f};
  if (k == 0) return a;
  if (k == 8) return mul_i<DIR>(a);
  const float c = C[k];
  // sin(k pi/16) = -cos((k+8) pi/16) for k < 8 and cos((k-8) pi/16) for k > 8
  const float s = DIR * C[(k + 8) & 15] * (k < 8 ? -1.f : 1.f);
  return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

// DFT_32 as 2 x 16 (decimation in time): E, O = DFT_16 of the even and odd inputs,
// X_k = E_k + w^k O_k, X_(k+16) = E_k - w^k O_k, w = exp(DIR 2 pi i / 32)
template <int DIR>
FR_HD void dft32(float2* v) {
  float2 e[16], o[16];
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    e[n] = v[2 * n];
    o[n] = v[2 * n + 1];
  }
  dft16<DIR>(e);
  dft16<DIR>(o);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float2 t = tw32<DIR>(o[k], k);
    v[k] = cadd(e[k], t);
    v[k + 16] = csub(e[k], t);
  }
}

// DFT_3: X_k = sum_n x_n w^(nk), w = exp(DIR 2 pi i / 3) = -1/2 + DIR i sqrt(3)/2
template <int DIR>
FR_HD void dft3(float2* v) {
  const float s3 = 0.86602540378443864676f;  // sin(2 pi / 3)
  const float2 a = v[0], sum = cadd(v[1], v[2]);
  const float2 m = make_float2(a.x - 0.5f * sum.x, a.y - 0.5f * sum.y);
  const float2 d = cscale(mul_i<DIR>(csub(v[1], v[2])), s3);
  v[0] = cadd(a, sum);
  v[1] = cadd(m, d);
  v[2] = csub(m, d);
}

// DFT_5 from the symmetric pairs (x1 + x4, x2 + x3) and antisymmetric pairs (x1 - x4, x2 - x3):
//   X_1,4 = x0 + c1 p1 + c2 p2 +- DIR i (s1 q1 + s2 q2)
//   X_2,3 = x0 + c2 p1 + c1 p2 +- DIR i (s2 q1 - s1 q2)
// with c_j = cos(2 pi j / 5), s_j = sin(2 pi j / 5)
template <int DIR>
FR_HD void dft5(float2* v) {
  const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
  const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
  const float2 x0 = v[0];
  const float2 p1 = cadd(v[1], v[4]), p2 = cadd(v[2], v[3]);
  const float2 q1 = csub(v[1], v[4]), q2 = csub(v[2], v[3]);
  const float2 a1 = make_float2(x0.x + c1 * p1.x + c2 * p2.x, x0.y + c1 * p1.y + c2 * p2.y);
  const float2 a2 = make_float2(x0.x + c2 * p1.x + c1 * p2.x, x0.y + c2 * p1.y + c1 * p2.y);
  const float2 b1 = mul_i<DIR>(make_float2(s1 * q1.x + s2 * q2.x, s1 * q1.y + s2 * q2.y));
  const float2 b2 = mul_i<DIR>(make_float2(s2 * q1.x - s1 * q2.x, s2 * q1.y - s1 * q2.y));
  v[0] = cadd(x0, cadd(p1, p2));
  v[1] = cadd(a1, b1);
  v[4] = csub(a1, b1);
  v[2] = cadd(a2, b2);
  v[3] = csub(a2, b2);
}

template <int R, int DIR>
FR_HD void dft_r(float2* v) {
  if constexpr (R == 3) {
    dft3<DIR>(v);
  } else if constexpr (R == 5) {
    dft5<DIR>(v);
  } else if constexpr (R == 2) {
    dft2<DIR>(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4<DIR>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    dft8<DIR>(v);
  } else if constexpr (R == 32) {
    dft32<DIR>(v);
  } else {
    static_assert(R == 16, "radix must be 2, 3, 4, 5, 8, 16 or 32");
    dft16<DIR>(v);
  }
}

// Radix schedule: log2 bits per stage, each at most 4 (radix 16).
// stage_bits(LOG2L, s) gives the bits of stage s (s = 0 first).
constexpr int num_stages(int log2l) { return (log2l + 3) / 4; }
constexpr int stage_bits(int log2l, int s) {
  // spread bits as evenly as possible, larger radices first
  return log2l / num_stages(log2l) + (s < (log2l % num_stages(log2l)) ? 1 : 0);
}
constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

// Mixed lengths L = c 2^k: the exponent k, the odd part c, its factors (5s first, then 3s) and
// the full stage schedule (odd stages, then the power-of-two schedule of 2^k).
constexpr int pow2_exp(int L) { return (L > 1 && (L & 1) == 0) ? 1 + pow2_exp(L >> 1) : 0; }
constexpr int odd_part(int L) { return L >> pow2_exp(L); }
constexpr int count_factor(int c, int f) { return (c > 1 && c % f == 0) ? 1 + count_factor(c / f, f) : 0; }
constexpr int strip_factor(int c, int f) { return (c > 1 && c % f == 0) ? strip_factor(c / f, f) : c; }
// lengths the pass kernels take: 16 | L (16 points per thread) and c a product of 3s and 5s
constexpr bool fft_length_ok(int L) {
  return L >= 16 && L % 16 == 0 && strip_factor(strip_factor(odd_part(L), 5), 3) == 1;
}
constexpr int odd_stages(int L) { return count_factor(odd_part(L), 5) + count_factor(odd_part(L), 3); }
// Schedules for P points per thread (16, or 32 for power-of-two lengths of at least 512): with
// P = 32 the power-of-two part opens with one radix-32 stage (8192 = 32 x 16 x 16: three stages
// instead of four of at most 16), with P = 16 every stage is of radix 16 or less.
constexpr int lead_bits(int L, int P) {
  return (P == 32 && odd_part(L) == 1 && pow2_exp(L) >= 9) ? 5 : 0;
}
constexpr int fft_num_stages(int L, int P = 16) {
  return odd_stages(L) + (lead_bits(L, P) ? 1 : 0) + num_stages(pow2_exp(L) - lead_bits(L, P));
}
constexpr int fft_radix(int L, int s, int P = 16) {
  return s < count_factor(odd_part(L), 5)                ? 5
         : s < odd_stages(L)                             ? 3
         : (lead_bits(L, P) > 0 && s == odd_stages(L))   ? (1 << lead_bits(L, P))
                                                         : 1 << stage_bits(pow2_exp(L) - lead_bits(L, P),
                                                                           s - odd_stages(L) - (lead_bits(L, P) ? 1 : 0));
}
constexpr int fft_ns_before(int L, int st, int P = 16) {
  return st == 0 ? 1 : fft_radix(L, st - 1, P) * fft_ns_before(L, st - 1, P);
}

// Shared-memory padding: one float2 of padding after every 16 elements breaks the
// power-of-two strides of the Stockham scatter.
FR_HD int spad(int i) { return i + (i >> 4); }
constexpr int spad_len(int n) { return n + (n >> 4); }

// v[r] *= w^r for r in [r, R), with w^r built from pw[e] = w^(2^e) and at most two more
// products per factor (a few ulp); all indices are compile-time, so everything stays in registers
template <int R, int r>
FR_HD void twiddle_rec(float2* v, const float2* pw, float2* wr) {
  if constexpr (r < R) {
    constexpr int h = ilog2(r);
    if constexpr (r == (1 << h))
      wr[r] = pw[h];
    else
      wr[r] = cmul(pw[h], wr[r - (1 << h)]);
    v[r] = cmul(v[r], wr[r]);
    twiddle_rec<R, r + 1>(v, pw, wr);
  }
}

FR_HD float2 ld_tw(const float2* p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}

// v[r] *= w^(r k), w = exp(DIR 2 pi i / (Ns R)) = tw[tstep] (conjugated for DIR = +1), tstep =
// L / (Ns R). Power-of-two radices build w^(r k) from the log2(R) entries w^(k 2^e) (a few
// ulp, log2(R) loads); radix 3 and 5 load their R - 1 entries tw[r k tstep] (r k tstep < L).
template <int R, int DIR>
FR_HD void apply_twiddles(float2* v, const float2* tw, int k, int tstep) {
  if constexpr ((R & (R - 1)) == 0) {
    constexpr int LB = ilog2(R);
    float2 pw[LB];
#pragma unroll
    for (int e = 0; e < LB; ++e) {
      float2 w = ld_tw(&tw[(k * tstep) << e]);
      if (DIR > 0) w.y = -w.y;
      pw[e] = w;
    }
    float2 wr[R];
    twiddle_rec<R, 1>(v, pw, wr);
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = ld_tw(&tw[r * k * tstep]);
      if (DIR > 0) w.y = -w.y;
      v[r] = cmul(v[r], w);
    }
  }
}

// One Stockham stage on a single task j, reading from `in` and writing to `out`
// (both indexed through spad), with the same twiddle construction as the kernels; used by the
// host emulation tests.
template <int R, int DIR>
FR_HD void stockham_task(const float2* in, float2* out, const float2* tw, int L, int Ns, int j) {
  float2 v[R];
  const int k = j % Ns;
  const int stride = L / R;
  const int tstep = L / (Ns * R);
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = in[spad(j + r * stride)];
  if (Ns > 1) apply_twiddles<R, DIR>(v, tw, k, tstep);
  dft_r<R, DIR>(v);
  const int base = (j / Ns) * Ns * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) out[spad(base + r * Ns)] = v[r];
}

}  // namespace fr
