// lise_ozaki.cuh -- FP64 spectral second derivative on the bf16 tensor cores.
//
// Along one axis of a periodic lattice of N points the kinetic operator of
// Sec. "Discretization", T = F^-1 [(alpha/2) k^2 F], is multiplication by the real
// symmetric circulant matrix
//   D2[n][k] = (1/N) sum_j (alpha/2) k_j^2 cos(k_j (n - k) a),
// so T applied to a block of lines is a matrix product with K = N.  The product
// is formed to FP64 accuracy from exact bf16 products (the splitting scheme of
// Ozaki, Ogita, Oishi and Rump, in its integer-digit form):
//   * every FP64 value of a group of lines sharing one binary exponent E (the
//     largest biased exponent in the group) becomes the integer
//       I = trunc(x 2^(1077 - E)),  |I| < 2^55,
//     written as 7 balanced base-256 digits I = sum_k d_k 256^(6-k), |d_k| <= 128;
//     the D2 entries likewise, with a common exponent (host tables);
//   * digit products are exact in bf16 x bf16 -> FP32, and the sum over K and
//     over all digit pairs (k, l) of one level L = k + l stays below 2^22, so each
//     level's FP32 accumulator holds an exact integer (checked at compile time);
//   * levels L <= 6 are kept (the dropped terms are below 2^-56 of the largest),
//     combined exactly in 64-bit integers and converted to FP64 with one rounding.
// The result agrees with the exact product to a few units of 2^-53 of the group's
// largest value, the accuracy class of an FP64 FFT.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lise {
namespace oz {

constexpr int S = 7;  // digits per value

// mma.sync m16n8k16, bf16 inputs, FP32 accumulate: c += a * b.
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}

// Biased binary exponent field of x (0 for zero and subnormals).
__device__ __forceinline__ unsigned exp_field(double x) {
  return ((unsigned)(__double_as_longlong(x) >> 52)) & 0x7FFu;
}

// bf16 bit pattern of a small integer (|d| <= 256): exact, through FP32
// (1.5 * 2^23 + d is exact in FP32 and its low bits are d).
__device__ __forceinline__ unsigned short bf16_of_int(int d) {
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
  return (unsigned short)(__float_as_uint(f) >> 16);
}

// bf16 bit pattern of (byte - 128) for the byte held in the low byte of w = 0x4B4000bb:
// as FP32 that word is 1.5 * 2^23 + byte, so one subtraction gives byte - 128 exactly.
__device__ __forceinline__ unsigned short bf16_of_biased_byte(unsigned w) {
  return (unsigned short)(__float_as_uint(__int_as_float(w) - 12583040.0f) >> 16);
}

// The 7 balanced base-256 digits (as bf16 bit patterns, most significant first)
// of I = trunc(x 2^(1077 - E)) (magnitude truncated), for E >= the exponent field
// of x (E >= 1).  Balanced digits without a carry chain: with the bias
// B = sum_{k=1..6} 128 * 256^(6-k), the low six bytes of I + B are d_k + 128 and
// (I + B) >> 48 is the top digit d_0.
__device__ __forceinline__ void split(double x, unsigned E, unsigned short d[S]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int s = (int)E - ex - 2;  // right shift of the 53-bit significand, >= -2
  unsigned long long u = s <= 0 ? (m << (-s)) : (s < 64 ? (m >> s) : 0ull);
  if (ex == 0) u = 0;
  const unsigned long long sm = (unsigned long long)((long long)b >> 63);  // 0, or all ones if x < 0
  const unsigned long long ib = ((u ^ sm) - sm) + 0x0000808080808080ull;   // I + B
  const unsigned lo = (unsigned)ib, hi = (unsigned)(ib >> 32);
  d[6] = bf16_of_biased_byte(__byte_perm(lo, 0x4B400000u, 0x7640));
  d[5] = bf16_of_biased_byte(__byte_perm(lo, 0x4B400000u, 0x7641));
  d[4] = bf16_of_biased_byte(__byte_perm(lo, 0x4B400000u, 0x7642));
  d[3] = bf16_of_biased_byte(__byte_perm(lo, 0x4B400000u, 0x7643));
  d[2] = bf16_of_biased_byte(__byte_perm(hi, 0x4B400000u, 0x7640));
  d[1] = bf16_of_biased_byte(__byte_perm(hi, 0x4B400000u, 0x7641));
  d[0] = bf16_of_int(((int)hi) >> 16);
}

// Exact FP32 integer (|v| < 2^22) to int.
__device__ __forceinline__ int f2i_exact(float v) { return __float_as_int(v + 12582912.0f) - 0x4B400000; }

// T = sum_L acc_L 2^(40 - 8 L) for L = 0..6 from the level sums (exact integers).
__device__ __forceinline__ long long combine(const int i[S]) {
  const int h1 = i[0] * 256 + i[1];
  const int h2 = i[2] * 256 + i[3];
  const int h3 = i[4] * 256 + i[5];
  return ((long long)h1 << 32) + ((long long)h2 << 16) + (long long)h3 + (long long)(i[6] >> 8);
}

// combine() from the FP32 bit patterns of (level + 1.5 * 2^23), i.e. before f2i_exact's
// subtraction: the bias cancels in 32-bit wrap-around arithmetic (each pair's true value
// 256 i_k + i_{k+1} fits in 31 bits), leaving one subtraction for the last level.
__device__ __forceinline__ long long combine_biased(const unsigned b[S]) {
  constexpr unsigned kM = 0x4B400000u, kM257 = 257u * kM;
  const int h1 = (int)(b[0] * 256u + b[1] - kM257);
  const int h2 = (int)(b[2] * 256u + b[3] - kM257);
  const int h3 = (int)(b[4] * 256u + b[5] - kM257);
  const int i6 = (int)(b[6] - kM);
  return ((long long)h1 << 32) + ((long long)h2 << 16) + (long long)h3 + (long long)(i6 >> 8);
}

// T * 2^sc rounded to FP64 (nearest even), integer operations only.
__device__ __forceinline__ double to_double(long long T, int sc) {
  if (T == 0) return 0.0;
  const unsigned long long sign = T < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long a = T < 0 ? (unsigned long long)(-T) : (unsigned long long)T;
  const int lz = __clzll((long long)a);
  a <<= lz;
  unsigned long long mant = a >> 11;
  const unsigned rem = (unsigned)(a & 0x7FFu);
  mant += (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
  int ex = 63 - lz + sc + 1023;
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  if (ex <= 0) return __longlong_as_double((long long)sign);
  return __longlong_as_double((long long)(sign | ((unsigned long long)ex << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// (T + Y) * 2^sc rounded to FP64, where y = Y * 2^sc is an FP64 value whose significand,
// aligned to the scale 2^sc, is truncated to an integer (bits below 2^sc dropped, as in
// the digit split); integer operations only.  Values of y above 2^(sc + 62) (not met by
// a kinetic term added to the same operator's other axes) fall back to an FP64 add.
__device__ __forceinline__ double add_to_double(long long T, double y, int sc) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const int ex = (int)((b >> 52) & 0x7FF);
  const int sh = ex - 1075 - sc;  // y = m 2^(ex - 1075) = (m 2^sh) 2^sc
  if (ex == 0x7FF || sh > 8) return to_double(T, sc) + y;
  const unsigned long long m = ex ? ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : 0ull;
  const unsigned long long u = sh >= 0 ? (m << sh) : (-sh < 64 ? (m >> -sh) : 0ull);
  const long long Y = (b >> 63) ? -(long long)u : (long long)u;
  return to_double(T + Y, sc);
}

// The same conversion through the FP64 unit (one I2F.F64 and an exponent add), for
// kernels whose FP64 pipe is otherwise idle; T * 2^sc must be a normal number.
__device__ __forceinline__ double to_double_hw(long long T, int sc) {
  if (T == 0) return 0.0;
  const double v = __ll2double_rn(T);
  return __longlong_as_double(__double_as_longlong(v) + ((long long)sc << 52));
}

// Output scale: value = T * 2^(sD + E - 1021) for a data group of exponent field E
// and D2 digits of I_D = round(D2 * 2^-sD).
__device__ __forceinline__ int out_scale(int sD, unsigned E) { return sD + (int)E - 1021; }

// Largest exponent field over a warp (sm_80+ warp reduction).
__device__ __forceinline__ unsigned warp_max(unsigned v) { return __reduce_max_sync(0xFFFFFFFFu, v); }

// One warp's product over all digit pairs of one output tile (16 data lines x 8
// output points): acc[L] (FP32, exact) += sum over pairs k + l = L of
// A_k (16 x K digits of the data, from shared memory) * B_l (K x 8, D2 digits in
// registers, b[l][ks][0..1]).  lda: byte offset function of the A tile.
// KS = K / 16.  When the per-level bound 7 K 2^14 reaches 2^22 the levels are
// converted to int after each k-step (iacc), else once at the end.
template <int KS, bool kTrans, typename AddrA>
__device__ __forceinline__ void tile_levels(int iacc[S][4], const uint32_t (&b)[S][KS][2], AddrA addr) {
  constexpr bool kPerStep = (7 * KS * 16 * 16384) >= (1 << 22);
#pragma unroll
  for (int L = 0; L < S; ++L)
#pragma unroll
    for (int e = 0; e < 4; ++e) iacc[L][e] = 0;
  float acc[S][4];
#pragma unroll
  for (int L = 0; L < S; ++L)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[L][e] = 0.f;
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      uint32_t a[4];
      if (kTrans)
        ldsm_x4_t(a, addr(k, ks));
      else
        ldsm_x4(a, addr(k, ks));
#pragma unroll
      for (int l = 0; l + k < S; ++l) mma16816(acc[k + l], a, b[l][ks]);
    }
    if (kPerStep) {
#pragma unroll
      for (int L = 0; L < S; ++L)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          iacc[L][e] += f2i_exact(acc[L][e]);
          acc[L][e] = 0.f;
        }
    }
  }
  if (!kPerStep) {
#pragma unroll
    for (int L = 0; L < S; ++L)
#pragma unroll
      for (int e = 0; e < 4; ++e) iacc[L][e] = f2i_exact(acc[L][e]);
  }
}

// D2 digit fragments of one 8-wide output tile nt for this lane, from the host
// table laid out [digit][nt][ks][lane][2] (uint32: two bf16, lower k in the low half).
template <int KS>
__device__ __forceinline__ void load_b(uint32_t (&b)[S][KS][2], const uint32_t* tab, int nt, int n_tiles) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int l = 0; l < S; ++l)
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const uint2 v = reinterpret_cast<const uint2*>(tab)[((l * n_tiles + nt) * KS + ks) * 32 + lane];
      b[l][ks][0] = v.x;
      b[l][ks][1] = v.y;
    }
}

}  // namespace oz
}  // namespace lise
