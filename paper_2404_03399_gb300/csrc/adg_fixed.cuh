// Fixed-point arithmetic of the integer composed step (adg_fixed.cu) and of the PE-face
// fix-up when it reads or writes fixed-point fields (adg_kernels.cu).
//
// On this part a warp's FP64 instruction occupies the FP64 pipe for 16 clocks (2 lanes per
// clock per SM) while a 32 x 32 -> 64-bit integer multiply-add issues at the integer rate,
// so the composed step (StepConsts) is evaluated in 58-bit block fixed point with integer
// multiplies (one scale per field and step; not exact: a sum of n terms is off by less than
// n/2 + 1/2 units of its last place, 2^-57 of the field's largest value per unit).
//
// Representation: a field at step n is either FP64 or int64 values X with one scale for the
// whole field, value = X 2^sigma (for a single instance the int64 values are the coordinates
// of each element in the block basis of Inst.Tb, with the headroom of Inst.fxh / fxe; the
// bounds below are those of nodal values, hb = he = 0). A step first brings its input to the working scale sigma'
// at which |X| < 2^57:
//   FP64 input: sigma' = En - 1079, En the largest biased FP64 exponent over u^n
//               (|x| < 2^(En - 1022)), X = round(x 2^-sigma');
//   int64 input (|X| < 2^62; b the bit length of the OR of all |X| less one for negative X,
//               so max |X| < 2^(b+1)): X' = round(X 2^-(b-56)), sigma' = sigma + (b - 56).
// Products split a value as X = xh 2^29 + xl with 0 <= xl < 2^29, and a coefficient c
// (|c| < 2) as C = round(c 2^58) = ch 2^29 + cl with balanced -2^28 <= cl < 2^28. Then
//   c x 2^-sigma' ~ C X 2^-58 = ch xh + (ch xl + cl xh) 2^-29 + cl xl 2^-58:
// the first two terms are three 32 x 32 -> 64-bit products that accumulate exactly in two
// 64-bit sums a and b; the last (|.| < 1/2 unit, with the sign of cl) is dropped. A sum of n
// terms is rounded once, a + round(b 2^-29): its error is below n/2 + 1/2 units, and the
// balanced coefficient limbs keep the dropped terms from all leaning one way (an unsigned cl
// would truncate every product downward). The host checks, per sum and from the
// coefficients, that a, b and the result stay inside 64 bits (every multiplicand below 2^58:
// inputs below 2^57, channel scalars below 2^58). Results are stored as int64 at sigma' or
// rounded to FP64 (round to nearest even).
//
// Scale bookkeeping: slot n % 3 of the instance's FxSlot[3] describes u^n: E (largest
// biased exponent when u^n is FP64; 2047 marks a NaN or infinity, carried through int64
// steps), sigma and mag (OR of |X|) when it is int64. Step n reads slot n % 3, raises slot
// (n + 1) % 3 and clears slot (n + 2) % 3 (block 0).
#pragma once

#include "adg_internal.h"

namespace adg {
namespace {

// b starts at 2^28, the rounding half-unit of fx_round.
struct FxAcc {
  long long a = 0, b = 1ll << 28;
};

// Each product is a 32 x 32 -> 64-bit mul.wide.s32 followed by a 64-bit add, which the
// assembler fuses into one wide multiply-add (measured: about one instruction per product; a
// PTX mad.wide.s32 came out near two and a half, a C++ (long long) product becomes a full
// 64-bit multiply, and forming the cross terms as high words of 32-bit products (mad.hi)
// issued more slowly than these wide products in this kernel's shape).
__device__ __forceinline__ long long fx_mul(int c, int x) {
  long long t;
  asm("mul.wide.s32 %0, %1, %2;" : "=l"(t) : "r"(c), "r"(x));
  return t;
}

// c = {ch, cl} (StepFixed limbs), x = (xh, xl) (fx_split).
__device__ __forceinline__ void fx_mac(FxAcc &s, int2 c, int xh, int xl) {
  s.a += fx_mul(c.x, xh);
  s.b += fx_mul(c.x, xl);
  s.b += fx_mul(c.y, xh);
}

__device__ __forceinline__ long long fx_round(const FxAcc &s) { return s.a + (s.b >> 29); }

// The 64-bit value with 32-bit halves lo, hi.
__device__ __forceinline__ long long fx_join(unsigned lo, unsigned hi) {
  long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
  return r;
}

// |X| < 2^58: xh = floor(X 2^-29), xl = X - xh 2^29 (two instructions; a balanced split
// of X measured 4% slower in the composed step).
__device__ __forceinline__ void fx_split(long long X, int &xh, int &xl) {
  xh = (int)(X >> 29);
  xl = (int)(X & 0x1FFFFFFF);
}

// FP64 -> int64 at scale sigma = En - 1079 (round half away from zero): |x| < 2^(En-1022)
// gives |X| < 2^57.
__device__ __forceinline__ long long fx_from_double(double x, int En) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)(((unsigned long long)bits >> 52) & 0x7ff);
  unsigned long long m = (unsigned long long)bits & 0xFFFFFFFFFFFFFull;
  int d = En - e;
  if (e) m |= 1ull << 52;
  else d -= 1;   // subnormal: the scale of exponent 1
  d = d < 0 ? 0 : (d > 63 ? 63 : d);
  m <<= 4;
  const unsigned long long M = (m + ((1ull << d) >> 1)) >> d;
  return bits < 0 ? -(long long)M : (long long)M;
}

// int64 at scale sigma -> FP64, round to nearest even; below the normal range the result
// is a signed zero, above it an infinity.
__device__ __forceinline__ double fx_to_double(long long y, int sigma) {
  if (y == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)y & 0x8000000000000000ull;
  const unsigned long long a = y < 0 ? 0ull - (unsigned long long)y : (unsigned long long)y;
  const int lz = __clzll((long long)a);
  const unsigned long long nrm = a << lz;
  unsigned long long m = nrm >> 11;
  const unsigned rem = (unsigned)nrm & 0x7ffu;
  m += (rem > 0x400u || (rem == 0x400u && (m & 1ull))) ? 1ull : 0ull;
  int ex = 1086 + sigma - lz;
  if (m >> 53) {
    m >>= 1;
    ++ex;
  }
  if (ex <= 0) return __longlong_as_double((long long)sgn);
  if (ex >= 2047) return __longlong_as_double((long long)(sgn | 0x7ff0000000000000ull));
  return __longlong_as_double(
      (long long)(sgn | ((unsigned long long)ex << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// int64 X at the stored scale -> working scale (shift = b - 57): rounded right shift when
// the field has grown past 2^57, exact left shift when it has shrunk.
__device__ __forceinline__ long long fx_rescale(long long X, int shift) {
  if (shift > 0) return (X + (1ll << (shift - 1))) >> shift;
  if (shift < 0) return (long long)((unsigned long long)X << (-shift));
  return X;
}

// x 2^e. Where 2^e is a normal FP64 number the product with it is the exactly scaled value,
// correctly rounded, as scalbn gives it; outside that range scalbn itself.
__device__ __forceinline__ double pow2_scale(double x, int e) {
  if ((unsigned)(e + 1022) <= 2045u) return x * __longlong_as_double((long long)(e + 1023) << 52);
  return scalbn(x, e);
}

__device__ __forceinline__ int biased_exponent(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
}

// A value whose bit length bounds that of |y| from below by at most one: |y| for y >= 0,
// |y| - 1 for y < 0 (the scale bookkeeping adds one bit of margin for it).
__device__ __forceinline__ unsigned long long fx_mag(long long y) {
  return (unsigned long long)(y ^ (y >> 63));
}

// Raises *slot to v unless it already holds at least v (slots only grow during a step, so
// a stale read can only cause a redundant atomic).
__device__ __forceinline__ void raise_slot(int *slot, int v) {
  if (v > *(volatile int *)slot) atomicMax(slot, v);
}

__device__ __forceinline__ void or_slot(unsigned long long *slot, unsigned long long v) {
  const unsigned long long cur = *(volatile unsigned long long *)slot;
  if ((cur | v) != cur) atomicOr(slot, v);
}

// Working scale of step n for input format fin (true: int64).
struct FxScale {
  int sigma;   // working scale sigma'
  int shift;   // int64 input: X' = fx_rescale(X, shift)
  int slot;    // n % 3
  bool bad;    // u^n holds a NaN or an infinity
};

// hb, he: the headroom of a block-basis state (Inst.fxh, Inst.fxe; 0 for nodal values):
// int64 inputs are brought below 2^(57 - hb), FP64 inputs converted at 2^(E - 1079 + he).
__device__ __forceinline__ FxScale fx_scale(const FxSlot *fx, int64_t n, bool fin, int hb = 0,
                                            int he = 0) {
  FxScale s;
  s.slot = (int)(n % 3);
  const FxSlot &cur = fx[s.slot];
  s.bad = cur.E >= 2047;
  if (!fin) {
    s.sigma = cur.E - 1079 + he;
    s.shift = 0;
  } else {
    const unsigned long long M = cur.mag;   // bit length of max |X| is at most b + 1
    s.shift = M ? (64 - __clzll((long long)M)) - 56 + hb : 0;
    s.sigma = cur.sigma + s.shift;
  }
  return s;
}

__device__ __forceinline__ int fx_next(int slot) { return slot == 2 ? 0 : slot + 1; }
__device__ __forceinline__ int fx_clear(int slot) { return slot == 0 ? 2 : slot - 1; }

}  // namespace
}  // namespace adg
