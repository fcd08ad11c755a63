// amrfd_device.cuh -- device-side building blocks of the FD-MP5 update.
//
// FP64 issue rate on GB300 is 1/64 of FP32, so everything that can be done
// exactly without the FP64 pipe is: comparisons, min/max, minmod, median and
// sign logic run on the integer pipe over the IEEE bit patterns (all exact), and
// the FP64 operations that remain are issued in the pipe's fastest form, DFMAs
// whose operands are all registers (see "FP64 operations as register FMAs").
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "amrfd_internal.h"

namespace amrfd {

enum { PH_EULER = 0, PH_MHD = 1 };

// Descriptor checks of the checked builds: a flux item lies inside its domain and its
// tile fits the shared-memory layout (P lines, SS doubles per line); a cell item lies
// inside its block.
__device__ __forceinline__ bool flux_item_ok(const DomDev* doms, int ndom, int ndim, int P, int SS,
                                             const FluxItem& it) {
  if (it.dom < 0 || it.dom >= ndom) return false;
  const DomDev& dm = doms[it.dom];
  const int d = it.d;
  if (d >= ndim || it.blk < 0 || it.blk >= dm.nb[0] * dm.nb[1] * dm.nb[2]) return false;
  const int od1 = d == 0 ? 1 : 0, od2 = d == 2 ? 1 : 2;
  const int bd = (d == 0 ? it.blk % dm.nb[0] : (d == 1 ? (it.blk / dm.nb[0]) % dm.nb[1] : it.blk / (dm.nb[0] * dm.nb[1])));
  return it.nl >= 1 && it.nl <= P && it.l0 >= 0 && it.l0 + it.nl <= dm.be[od1] * dm.be[od2] && it.s0 >= 0 &&
         it.slen >= 1 && it.slen + 2 * kGhost <= SS && bd * dm.be[d] + it.s0 + it.slen <= dm.n[d];
}

__device__ __forceinline__ bool cell_item_ok(const DomDev* doms, int ndom, const CellItem& ci) {
  if (ci.dom < 0 || ci.dom >= ndom) return false;
  const DomDev& dm = doms[ci.dom];
  return ci.blk >= 0 && ci.blk < dm.nb[0] * dm.nb[1] * dm.nb[2] && ci.c0 >= 0 && ci.cnt >= 0 &&
         ci.c0 + ci.cnt <= dm.be[0] * dm.be[1] * dm.be[2];
}

// ---------------------------------------------------------------- exact helpers
// Bit pattern of x through an opaque PTX move, so that integer tests on it stay on the
// integer pipe (from a plain reinterpretation the compiler rebuilds FP64 compares,
// absolute values and negations).
__device__ __forceinline__ long long dbits(double x) {
  long long r;
  asm("mov.b64 %0, %1;" : "=l"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double bitsd(long long b) { return __longlong_as_double(b); }

// The helpers below are written in inline PTX so that they stay on the integer
// pipe: left to itself the compiler turns some of these bit manipulations of
// doubles back into FP64 compares, negations or multiplies.

// Monotone signed-integer key of a double (total order; -0 sorts before +0).
// Bit pattern of |x| (in PTX: masking the sign of a double's bits in C++ is turned by
// the compiler into an FP64 add with an absolute-value operand).
__device__ __forceinline__ long long abits(double x) {
  long long r;
  asm("{\n\t.reg .b64 t;\n\tmov.b64 t, %1;\n\tand.b64 %0, t, 0x7fffffffffffffff;\n\t}" : "=l"(r) : "d"(x));
  return r;
}

// Sign bit of x as 0/1 (in PTX, for the same reason).
__device__ __forceinline__ unsigned sbit(double x) {
  unsigned r;
  asm("{\n\t.reg .b64 t;\n\tmov.b64 t, %1;\n\tshr.u64 t, t, 63;\n\tcvt.u32.u64 %0, t;\n\t}" : "=r"(r) : "d"(x));
  return r;
}

__device__ __forceinline__ long long okey(double x) {
  long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

#define AMRFD_OKEY(dst, src) \
  "shr.s64 " dst ", " src ", 63;\n\t" "and.b64 " dst ", " dst ", 0x7fffffffffffffff;\n\t" \
  "xor.b64 " dst ", " src ", " dst ";\n\t"

__device__ __forceinline__ double imin(double a, double b) {
  double r;
  asm("{\n\t.reg .b64 xa, xb, ka, kb;\n\t.reg .pred p;\n\t"
      "mov.b64 xa, %1;\n\tmov.b64 xb, %2;\n\t" AMRFD_OKEY("ka", "xa") AMRFD_OKEY("kb", "xb")
      "setp.lt.s64 p, ka, kb;\n\tselp.b64 xa, xa, xb, p;\n\tmov.b64 %0, xa;\n\t}"
      : "=d"(r) : "d"(a), "d"(b));
  return r;
}
__device__ __forceinline__ double imax(double a, double b) {
  double r;
  asm("{\n\t.reg .b64 xa, xb, ka, kb;\n\t.reg .pred p;\n\t"
      "mov.b64 xa, %1;\n\tmov.b64 xb, %2;\n\t" AMRFD_OKEY("ka", "xa") AMRFD_OKEY("kb", "xb")
      "setp.lt.s64 p, ka, kb;\n\tselp.b64 xa, xb, xa, p;\n\tmov.b64 %0, xa;\n\t}"
      : "=d"(r) : "d"(a), "d"(b));
  return r;
}

// minmod(a,b) = (sgn a + sgn b)/2 * min(|a|,|b|): the smaller-magnitude argument
// when both have the same sign, else zero.
__device__ __forceinline__ double iminmod(double a, double b) {
  double r;
  asm("{\n\t.reg .b64 xa, xb, ma, mb, t;\n\t.reg .pred p, q;\n\t"
      "mov.b64 xa, %1;\n\tmov.b64 xb, %2;\n\t"
      "and.b64 ma, xa, 0x7fffffffffffffff;\n\tand.b64 mb, xb, 0x7fffffffffffffff;\n\t"
      "setp.lt.u64 p, ma, mb;\n\tselp.b64 t, xa, xb, p;\n\t"
      "xor.b64 ma, xa, xb;\n\tsetp.lt.s64 q, ma, 0;\n\tselp.b64 t, 0, t, q;\n\t"
      "mov.b64 %0, t;\n\t}"
      : "=d"(r) : "d"(a), "d"(b));
  return r;
}

// median(x, y, z) -- one of its arguments, no rounding
__device__ __forceinline__ double imedian(double x, double y, double z) {
  return imax(imin(x, y), imin(imax(x, y), z));
}

// x <= c for a finite non-negative constant c (NaN compares false)
__device__ __forceinline__ bool ile_pos(double x, double c) {
  unsigned r;
  asm("{\n\t.reg .b64 xa, xc, ka;\n\t.reg .pred p;\n\t"
      "mov.b64 xa, %1;\n\tmov.b64 xc, %2;\n\t" AMRFD_OKEY("ka", "xa")
      "setp.le.s64 p, ka, xc;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r) : "d"(x), "d"(c));
  return r != 0;
}

// x * 2^K exactly. The exponent field is adjusted on the integer pipe when the
// result stays a normal number (or x is +-0); otherwise (subnormal or near-overflow
// input, never met in practice) one FP64 multiply in an out-of-line call.
static __device__ __noinline__ double dscale_slow(double x, double f) { return x * f; }

template <int K>
__device__ __forceinline__ double dscale(double x) {
  double r;
  unsigned ok;
  constexpr long long inc = (long long)K << 52;
  constexpr long long lo = (long long)(1 + (K < 0 ? -K : 0)) << 52;   // smallest exponent field allowed
  constexpr long long hi = (long long)(2046 - (K > 0 ? K : 0)) << 52;  // largest exponent field allowed
  asm("{\n\t.reg .b64 xa, m, e, y;\n\t.reg .pred pz, plo, phi, pok;\n\t"
      "mov.b64 xa, %2;\n\t"
      "and.b64 m, xa, 0x7fffffffffffffff;\n\t"
      "and.b64 e, xa, 0x7ff0000000000000;\n\t"
      "setp.eq.s64 pz, m, 0;\n\t"
      "setp.ge.s64 plo, e, %3;\n\t"
      "setp.le.s64 phi, e, %4;\n\t"
      "and.pred pok, plo, phi;\n\t"
      "or.pred pok, pok, pz;\n\t"
      "add.s64 y, xa, %5;\n\t"
      "selp.b64 y, xa, y, pz;\n\t"
      "mov.b64 %0, y;\n\t"
      "selp.u32 %1, 1, 0, pok;\n\t}"
      : "=d"(r), "=r"(ok) : "d"(x), "l"(lo), "l"(hi), "l"(inc));
  if (__builtin_expect(ok == 0, 0)) r = dscale_slow(x, K >= 0 ? (double)(1LL << (K >= 0 ? K : 0)) : 1.0 / (double)(1LL << (K < 0 ? -K : 0)));
  return r;
}

// -x by flipping the sign bit (in PTX: the compiler would otherwise emit an FP64 add)
__device__ __forceinline__ double dneg(double x) {
  double r;
  asm("{\n\t.reg .b64 t;\n\tmov.b64 t, %1;\n\txor.b64 t, t, 0x8000000000000000;\n\tmov.b64 %0, t;\n\t}"
      : "=d"(r) : "d"(x));
  return r;
}

// |x| rounded toward zero to FP32, from the bits of |x| whose exponent lies in
// [2^-60, 2^61) (caller checks): the mantissa's top 23 bits and a rebiased exponent.
__device__ __forceinline__ float f32_trunc_abs(long long ax) {
  float r;
  asm("{\n\t.reg .b64 t;\n\t.reg .b32 u;\n\t"
      "shr.u64 t, %1, 29;\n\tsub.u64 t, t, 7516192768;\n\tcvt.u32.u64 u, t;\n\tmov.b32 %0, u;\n\t}"
      : "=f"(r) : "l"(ax));
  return r;
}

// FP64 evaluation of the acceptance test, out of line so that it costs nothing
// unless taken.
static __device__ __noinline__ bool mp_accept_slow(double X, double mp, double eps) {
  return ile_pos(X * (X - mp), eps);
}

// The MP acceptance test fl(X * fl(X - mp)) <= eps, decided exactly as the FP64
// expression decides it. Signs are read from the bit patterns; a product of
// like-signed factors is estimated in FP32 with a rigorous error bound (inputs
// truncated to 23 bits, three FP32 roundings, the two FP64 roundings), and only
// an estimate within the bound of eps falls back to the FP64 evaluation.
__device__ __forceinline__ bool mp_accept(double X, double mp, double eps) {
  long long ax, am;
  unsigned quick, opp;
  // sign analysis on the bit patterns: X = +-0 (product +-0), X == mp (zero
  // difference), or X and X - mp of opposite sign (product <= 0) accept at once
  asm("{\n\t.reg .b64 bx, bm, kx, km;\n\t.reg .pred p, q, r;\n\t"
      "mov.b64 bx, %4;\n\tmov.b64 bm, %5;\n\t"
      "and.b64 %0, bx, 0x7fffffffffffffff;\n\tand.b64 %1, bm, 0x7fffffffffffffff;\n\t"
      AMRFD_OKEY("kx", "bx") AMRFD_OKEY("km", "bm")
      "setp.eq.s64 p, %0, 0;\n\tsetp.eq.s64 q, kx, km;\n\tor.pred p, p, q;\n\t"
      "setp.gt.s64 q, kx, km;\n\tsetp.ge.s64 r, bx, 0;\n\txor.pred q, q, r;\n\tor.pred p, p, q;\n\t"
      "selp.u32 %2, 1, 0, p;\n\t"
      "xor.b64 kx, bx, bm;\n\tsetp.lt.s64 q, kx, 0;\n\tselp.u32 %3, 1, 0, q;\n\t}"
      : "=l"(ax), "=l"(am), "=r"(quick), "=r"(opp) : "d"(X), "d"(mp));
  if (quick) return true;
  const int ex = (int)(ax >> 52), em = (int)(am >> 52);
  // |X|, |mp| < 2^-60: fl(X - mp) <= 2^-59 and the product is at most 2^-119
  if (ex < 963 && em < 963 && dbits(eps) >= (904LL << 52)) return true;
  const bool in_range = ex >= 963 && ex <= 1083 && (am == 0 || (em >= 963 && em <= 1083));
  if (in_range) {
    const float fx = f32_trunc_abs(ax);
    const float fm0 = am == 0 ? 0.0f : f32_trunc_abs(am);
    // |X - mp| = |X| - s mp with s = sign(X): the subtrahend keeps its magnitude, its
    // sign is flipped when mp and X have opposite signs
    const float fm = opp ? -fm0 : fm0;
    const float df = fx - fm;
    const float pe = fx * df;
    const float bound = 9.5367431640625e-07f * fmaf(fx, fx + fabsf(fm), fabsf(pe));  // 2^-20 (...)
    const float ef = (float)eps;
    if (pe + bound < ef * 0.99999809f) return true;   // ef (1 - 2^-19)
    if (pe - bound > ef * 1.00000191f) return false;  // ef (1 + 2^-19)
  }
  return mp_accept_slow(X, mp, eps);
}

// ------------------------------------------------ FP64 operations as register FMAs
// GB300 issues a DFMA whose three operands are registers at 19.6 G warp instructions/s,
// and a DADD, a DMUL or a DFMA with an immediate or constant-bank operand at 16.5 G/s
// (independent chains on every SM, whatever the operand values). The hot loops therefore
// form sums, differences and products as register DFMAs, bit for bit the plain
// operations: x + y = fma(x, 1, y) and x - y = fma(x, 1, -y) (the exact sum, rounded
// once), c x = fma(c, x, -0) (adding -0 changes no product, zeros included). The
// constants are read from a mutable device array through an opaque load, so the
// compiler can neither fold them back into immediates nor read them from the constant
// bank.
enum { K_ONE, K_MZ, K_HALF, K_C22, K_C4, K_C48, K_C6, K_ZERO, K_C26, K_C54, K_C83, K_TWO, K_THIRD, K_C16, K_COUNT };
static __device__ double g_regk[K_COUNT] = {1.0, -0.0, 0.5, 22.0 / 60.0, 4.0 / 60.0, 48.0 / 60.0, 6.0 / 60.0, 0.0,
                                            26.0 / 60.0, 54.0 / 60.0, 8.0 / 3.0, 2.0, 1.0 / 3.0, 1.6};

// Constant K_* as a register value (an opaque load at this point of the code).
__device__ __forceinline__ double ldk(int i) {
  double x;
  asm volatile("ld.f64 %0, [%1];" : "=d"(x) : "l"(g_regk + i));
  return x;
}

__device__ __forceinline__ double radd(double x, double y, double one) { return fma(x, one, y); }
__device__ __forceinline__ double rsub(double x, double y, double one) { return fma(x, one, -y); }
__device__ __forceinline__ double rmul(double c, double x, double mz) { return fma(c, x, mz); }

// 2 (f_or - f_i) of MP5 from the differences: (-4 Dm + 22 D0 + 48 D1 - 6 Dp) / 60, mirrored
// (all signs flipped) for NEG; every sweep forms it with this one operation order. The
// weights are loaded where they are used, which keeps them out of the sweep's registers.
template <bool NEG>
__device__ __forceinline__ double mp5_x(double Dm, double D0, double D1, double Dp) {
  const double mz = ldk(K_MZ), c22 = ldk(K_C22), c4 = ldk(K_C4), c48 = ldk(K_C48), c6 = ldk(K_C6);
  const double x0 = fma(NEG ? -c22 : c22, D0, mz);
  const double x1 = fma(NEG ? c4 : -c4, Dm, x0);
  const double x2 = fma(NEG ? -c48 : c48, D1, x1);
  return fma(NEG ? c6 : -c6, Dp, x2);
}

// minmod4(4 ka - kb, 4 kb - ka, ka, kb): the curvature-limited second difference at
// a face from the curvatures of its two cells. Zero unless ka, kb share a sign; then,
// with s the smaller and l the larger in magnitude, 4 l - s never wins and the
// result is 4 s - l if it keeps the sign and is smaller than s, else s (one FMA).
// Selections and the sign flip of l are integer operations.
__device__ __forceinline__ double dm4(double ka, double kb) {
  double sm, nl;
  unsigned same;
  asm("{\n\t.reg .b64 a, b, ma, mb, s, l, t;\n\t.reg .pred p, q, z;\n\t"
      "mov.b64 a, %3;\n\tmov.b64 b, %4;\n\t"
      "and.b64 ma, a, 0x7fffffffffffffff;\n\tand.b64 mb, b, 0x7fffffffffffffff;\n\t"
      "setp.lt.u64 p, ma, mb;\n\t"
      "selp.b64 s, a, b, p;\n\tselp.b64 l, b, a, p;\n\t"
      "xor.b64 l, l, 0x8000000000000000;\n\t"
      "xor.b64 t, a, b;\n\tsetp.ge.s64 q, t, 0;\n\t"
      "setp.ne.s64 z, ma, 0;\n\tand.pred q, q, z;\n\t"
      "setp.ne.s64 z, mb, 0;\n\tand.pred q, q, z;\n\t"
      "mov.b64 %0, s;\n\tmov.b64 %1, l;\n\tselp.u32 %2, 1, 0, q;\n\t}"
      : "=d"(sm), "=d"(nl), "=r"(same) : "d"(ka), "d"(kb));
  if (!same) return 0.0;
  const double t = fma(4.0, sm, nl);
  double r;
  asm("{\n\t.reg .b64 s, t, ms, mt, x;\n\t.reg .pred p, q;\n\t"
      "mov.b64 s, %1;\n\tmov.b64 t, %2;\n\t"
      "and.b64 ms, s, 0x7fffffffffffffff;\n\tand.b64 mt, t, 0x7fffffffffffffff;\n\t"
      "setp.lt.u64 p, mt, ms;\n\tselp.b64 x, t, s, p;\n\t"
      "xor.b64 ms, s, t;\n\tsetp.lt.s64 q, ms, 0;\n\t"
      "setp.eq.s64 p, mt, 0;\n\tor.pred q, q, p;\n\t"
      "selp.b64 x, 0, x, q;\n\tmov.b64 %0, x;\n\t}"
      : "=d"(r) : "d"(sm), "d"(t));
  return r;
}

// ---------------------------------------------------------- MP5 in difference form
// MP5 (Suresh & Huynh 1997) at face i+1/2 from (f_{i-2}, ..., f_{i+2}), written in
// differences Dm = f_{i-1}-f_{i-2}, D0 = f_i-f_{i-1}, D1 = f_{i+1}-f_i, Dp = f_{i+2}-f_{i+1}
// and the curvature-limited second differences Mp (at i+1/2) and Mm (at i-1/2):
//   f_or - f_i = (11 D0 - 2 Dm + 24 D1 - 3 Dp)/60,  f_mp - f_i = minmod(D1, 4 D0),
//   f_ul - f_i = 4 D0,  f_md - f_i = D1/2 - Mp/2,  f_lc - f_i = D0/2 + 4 Mm/3,
// with the acceptance test (f_or - f_i)(f_or - f_mp) <= eps and otherwise
// median(f_or, f_min, f_max). Everything is carried at twice its value, which makes
// the halvings and the factor 4 exact exponent shifts; the result is
// 2 (f_face - f_i). NEG evaluates the mirror-image stencil whose differences are
// the negatives of the ones passed in (the right-biased reconstruction).
// eps16 = 16 eps: 4 eps for values doubled twice (splitting without the 1/2, and here).
//
// mp5_rel2_r also reports whether the acceptance test failed (rej). CARRY takes the
// curvature-limited second differences Mp, Mm from the caller (carried along the line);
// otherwise they are formed here, only when the test fails, from the curvatures of cells
// i-1, i, i+1 with the operands and order of the carried ones (for NEG, of the mirrored
// stencil), so both forms give the same result.
template <bool NEG, bool CARRY>
__device__ __forceinline__ double mp5_rel2_r(double Dm, double D0, double D1, double Dp, double Mp, double Mm,
                                             double eps16, bool& rej, double one) {
  const double X = mp5_x<NEG>(Dm, D0, D1, Dp);  // 2 (f_or - f_i)
  const double d0 = NEG ? dneg(D0) : D0;
  const double d1 = NEG ? dneg(D1) : D1;
  const double ul = dscale<3>(d0);     // 2 (f_ul - f_i)
  const double d1x2 = dscale<1>(d1);   // 2 (f_{i+1} - f_i)
  const double mp = iminmod(d1x2, ul);  // 2 (f_mp - f_i)
  rej = false;
  if (mp_accept(X, mp, eps16)) return X;
  rej = true;
  if (!CARRY) {
    if (!NEG) {
      const double k0 = rsub(D1, D0, one);
      Mp = dm4(k0, rsub(Dp, D1, one));
      Mm = dm4(rsub(D0, Dm, one), k0);
    } else {
      const double k0 = rsub(D0, D1, one);
      Mp = dm4(rsub(D1, Dp, one), k0);
      Mm = dm4(k0, rsub(Dm, D0, one));
    }
  }
  const double md = rsub(d1, Mp, one);          // 2 (f_md - f_i)
  const double lc = fma(ldk(K_C83), Mm, d0);    // 2 (f_lc - f_i)
  const double fmin = imax(imin(imin(0.0, d1x2), md), imin(imin(0.0, ul), lc));
  const double fmax = imin(imax(imax(0.0, d1x2), md), imax(imax(0.0, ul), lc));
  return imedian(X, fmin, fmax);
}

// ------------------------------------------------ selection-tracking variants
// The same operations as mp5_rel2_r / dm4 (bit-identical results), also reporting
// which linear piece produced the value, for the discrete adjoint.
enum { SEL_X = 0, SEL_ZERO = 1, SEL_D1 = 2, SEL_MD = 3, SEL_UL = 4, SEL_LC = 5 };

__device__ __forceinline__ void imin_sel(double a, int ca, double b, int cb, double& r, int& cr) {
  const bool t = okey(a) < okey(b);
  r = t ? a : b;
  cr = t ? ca : cb;
}
__device__ __forceinline__ void imax_sel(double a, int ca, double b, int cb, double& r, int& cr) {
  const bool t = okey(a) < okey(b);
  r = t ? b : a;
  cr = t ? cb : ca;
}

// Gradient of the MP5 value (mp5_rel2_r) w.r.t. (Dm, D0, D1, Dp, Mp, Mm) for the piece `code`, times g.
template <bool NEG>
__device__ __forceinline__ void mp5_rel2_grad(int code, double g, double& gDm, double& gD0, double& gD1,
                                              double& gDp, double& gMp, double& gMm) {
  constexpr double sg = NEG ? -1.0 : 1.0;
  gDm = gD0 = gD1 = gDp = gMp = gMm = 0.0;
  switch (code) {
    case SEL_X:
      gDm = (-sg * (4.0 / 60.0)) * g;
      gD0 = (sg * (22.0 / 60.0)) * g;
      gD1 = (sg * (48.0 / 60.0)) * g;
      gDp = (-sg * (6.0 / 60.0)) * g;
      break;
    case SEL_D1: gD1 = (2.0 * sg) * g; break;
    case SEL_MD: gD1 = sg * g; gMp = -g; break;
    case SEL_UL: gD0 = (8.0 * sg) * g; break;
    case SEL_LC: gD0 = sg * g; gMm = (8.0 / 3.0) * g; break;
    default: break;
  }
}

// dm4 with the chosen piece: 0 zero, 1 ka, 2 kb, 3 4 ka - kb, 4 4 kb - ka.
__device__ __forceinline__ double dm4_sel(double ka, double kb, int& code) {
  const long long a = dbits(ka), b = dbits(kb);
  const long long M = 0x7fffffffffffffffLL;
  const long long ma = a & M, mb = b & M;
  code = 0;
  if (((a ^ b) < 0) | (ma == 0) | (mb == 0)) return 0.0;
  const bool as = ma < mb;
  const double sm = as ? ka : kb, lg = as ? kb : ka;
  const long long ms = as ? ma : mb;
  const double t = fma(4.0, sm, -lg);
  const long long bt = dbits(t);
  if (((bt ^ dbits(sm)) < 0) | ((bt & M) == 0)) return 0.0;
  if ((bt & M) < ms) { code = as ? 3 : 4; return t; }
  code = as ? 1 : 2;
  return sm;
}

__device__ __forceinline__ void dm4_grad(int code, double g, double& gka, double& gkb) {
  gka = gkb = 0.0;
  if (code == 1) gka = g;
  else if (code == 2) gkb = g;
  else if (code == 3) { gka = 4.0 * g; gkb = -g; }
  else if (code == 4) { gkb = 4.0 * g; gka = -g; }
}

// mp5_rel2_r without CARRY (bit-identical value) that also records the pieces taken: the
// curvature-limited second differences are formed only where the acceptance test fails,
// with dm4_sel, and the median's selections are tracked. rec = piece of the value | piece
// of Mp << 3 | piece of Mm << 6 (the curvature pieces are 0 where the value is f_or,
// which reads neither).
template <bool NEG>
__device__ __forceinline__ double mp5_rel2_rec(double Dm, double D0, double D1, double Dp, double eps16, int& rec,
                                               double one) {
  const double X = mp5_x<NEG>(Dm, D0, D1, Dp);
  const double d0 = NEG ? dneg(D0) : D0;
  const double d1 = NEG ? dneg(D1) : D1;
  const double ul = dscale<3>(d0);
  const double d1x2 = dscale<1>(d1);
  const double mp = iminmod(d1x2, ul);
  rec = SEL_X;
  if (mp_accept(X, mp, eps16)) return X;
  double Mp, Mm;
  int cp, cm;
  if (!NEG) {
    const double k0 = rsub(D1, D0, one);
    Mp = dm4_sel(k0, rsub(Dp, D1, one), cp);
    Mm = dm4_sel(rsub(D0, Dm, one), k0, cm);
  } else {
    const double k0 = rsub(D0, D1, one);
    Mp = dm4_sel(rsub(D1, Dp, one), k0, cp);
    Mm = dm4_sel(k0, rsub(Dm, D0, one), cm);
  }
  const double md = rsub(d1, Mp, one);
  const double lc = fma(ldk(K_C83), Mm, d0);
  double a, b, fmin, fmax, t1, t2, t3;
  int ca, cb, cmin, cmax, c1, c2, c3;
  imin_sel(0.0, SEL_ZERO, d1x2, SEL_D1, a, ca);
  imin_sel(a, ca, md, SEL_MD, a, ca);
  imin_sel(0.0, SEL_ZERO, ul, SEL_UL, b, cb);
  imin_sel(b, cb, lc, SEL_LC, b, cb);
  imax_sel(a, ca, b, cb, fmin, cmin);
  imax_sel(0.0, SEL_ZERO, d1x2, SEL_D1, a, ca);
  imax_sel(a, ca, md, SEL_MD, a, ca);
  imax_sel(0.0, SEL_ZERO, ul, SEL_UL, b, cb);
  imax_sel(b, cb, lc, SEL_LC, b, cb);
  imin_sel(a, ca, b, cb, fmax, cmax);
  imin_sel(X, SEL_X, fmin, cmin, t1, c1);
  imax_sel(X, SEL_X, fmin, cmin, t2, c2);
  imin_sel(t2, c2, fmax, cmax, t3, c3);
  double r;
  int code;
  imax_sel(t1, c1, t3, c3, r, code);
  rec = code | (cp << 3) | (cm << 6);
  return r;
}

// Reciprocal of a positive normal double: FP32 seed from the leading bits (integer
// conversion, MUFU reciprocal) and two Newton steps y <- y + y (1 - x y) in FP64.
__device__ __forceinline__ double frcp(double x) {
  const long long b = dbits(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e < 1023 - 120 || e > 1023 + 120) return 1.0 / x;
  const unsigned fb = ((unsigned)((unsigned long long)b >> 32) & 0x80000000u) | ((unsigned)(e - 1023 + 127) << 23) |
                      (unsigned)((b >> 29) & 0x7fffff);
  const unsigned yb = __float_as_uint(__frcp_rn(__uint_as_float(fb)));
  const long long db = ((long long)(yb & 0x80000000u) << 32) | ((long long)(((yb >> 23) & 0xff) - 127 + 1023) << 52) |
                       ((long long)(yb & 0x7fffff) << 29);
  double y = bitsd(db);
  const double one = ldk(K_ONE);
  double r = fma(-x, y, one);
  y = fma(y, r, y);
  r = fma(-x, y, one);
  return fma(y, r, y);
}

// ------------------------------------------------- exact characteristic speeds
// Same operation order as the CPU definition (no contraction), so that splitting
// speeds and time steps of a given state agree bit for bit.
struct Prim {
  double rho, v[3], p, B[3], psi;
};

template <int PHYS, int NV>
__device__ __forceinline__ bool cons2prim_exact(const double* u, double gamma, int ndim, Prim& w) {
  w.rho = u[0];
  const int nm = PHYS == PH_EULER ? NV - 2 : 3;
#pragma unroll
  for (int k = 0; k < 3; k++) w.v[k] = (k < nm) ? __ddiv_rn(u[1 + k], w.rho) : 0.0;
  double vv = __dadd_rn(__dadd_rn(__dmul_rn(w.v[0], w.v[0]), __dmul_rn(w.v[1], w.v[1])), __dmul_rn(w.v[2], w.v[2]));
  double ekin = __dmul_rn(__dmul_rn(0.5, w.rho), vv);
  double emag = 0.0, E;
  if (PHYS == PH_MHD) {
    w.B[0] = u[5]; w.B[1] = u[6]; w.B[2] = u[7]; w.psi = u[8];
    emag = __dmul_rn(0.5, __dadd_rn(__dadd_rn(__dmul_rn(w.B[0], w.B[0]), __dmul_rn(w.B[1], w.B[1])),
                                    __dmul_rn(w.B[2], w.B[2])));
    E = u[4];
  } else {
    w.B[0] = w.B[1] = w.B[2] = 0.0; w.psi = 0.0;
    E = u[NV - 1];
  }
  w.p = __dmul_rn(__dsub_rn(gamma, 1.0), __dsub_rn(__dsub_rn(E, ekin), emag));
  return (w.rho > 0.0) && (w.p > 0.0) && isfinite(w.rho) && isfinite(w.p) && isfinite(w.psi);
}

template <int PHYS>
__device__ __forceinline__ double char_speed_exact(const Prim& w, double gamma, int d) {
  if (PHYS == PH_EULER) return __dadd_rn(fabs(w.v[d]), __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, w.p), w.rho)));
  double a2 = __ddiv_rn(__dmul_rn(gamma, w.p), w.rho);
  double b2 = __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(w.B[0], w.B[0]), __dmul_rn(w.B[1], w.B[1])),
                                  __dmul_rn(w.B[2], w.B[2])), w.rho);
  double s = __dadd_rn(a2, b2);
  double bd = w.B[d];
  double disc = __dsub_rn(__dmul_rn(s, s), __ddiv_rn(__dmul_rn(__dmul_rn(4.0, a2), __dmul_rn(bd, bd)), w.rho));
  if (disc < 0.0) disc = 0.0;
  double cf = __dsqrt_rn(__dmul_rn(0.5, __dadd_rn(s, __dsqrt_rn(disc))));
  return __dadd_rn(fabs(w.v[d]), cf);
}

// --------------------------------------- bounded FP32 estimate of the speeds
// FP32 conversion of x (truncation, relative error < 2^-23) when |x| lies in
// [2^-100, 2^100] or x is zero; ok = false otherwise.
__device__ __forceinline__ float f32_of(double x, bool& ok) {
  const long long ax = abits(x);
  if (ax == 0) return 0.0f;
  const int e = (int)(ax >> 52);
  if (e < 923 || e > 1123) { ok = false; return 0.0f; }
  const float f = f32_trunc_abs(ax);
  return ax != dbits(x) ? -f : f;
}

// As f32_of for a momentum or field component, except that a nonzero |x| < 2^-100
// gives 0 and sets flushed (the caller bounds the effect of the change).
__device__ __forceinline__ float f32_of_flush(double x, bool& ok, bool& flushed) {
  const long long ax = abits(x);
  if (ax == 0) return 0.0f;
  const int e = (int)(ax >> 52);
  if (e < 923) { flushed = true; return 0.0f; }
  if (e > 1123) { ok = false; return 0.0f; }
  const float f = f32_trunc_abs(ax);
  return ax != dbits(x) ? -f : f;
}

// Bounds lo <= c_d <= up of the exact characteristic speeds of a cell (d < ndim), and
// of its CFL rate sum_d c_d/dx_d (index 3), from an FP32 evaluation. The relative
// error of every FP32 quantity is bounded by the input truncation (2^-23 each), the
// FP32 roundings (2^-24 each) and the cancellation in p = (gamma-1)(E - rho v^2/2 -
// B^2/2), which scales them by T/S with T = E + rho v^2/2 + B^2/2, S = p/(gamma-1);
// the discriminant of the fast speed is formed as (a^2 - b_d^2)^2 + b_t^2 (b_t^2 +
// 2 (a^2 + b_d^2)) (b_t the transverse Alfven speed), a sum of non-negative terms,
// so the square roots do not amplify it. The bound used, 2^-17 (T/S + 1), holds with
// a margin of four. Momentum and field components below 2^-100 in magnitude (the
// exactly-zero components of a uniform state pick up such values ahead of a wave)
// enter as 0. Each such change moves c_d = |v_d| + c_f by at most 2^-100 (1.5 +
// gamma) (1/rho + 1/sqrt(rho)): c_f is 1-Lipschitz in the sound speed a and in
// b_d = |B_d|/sqrt(rho), 1.5-Lipschitz in the transverse b_t, and a moves by at most
// the square root of the change of a^2. With at most six such components, with
// T/S < 2^10 (FP32 a^2 then within 2^-10 of its value) and with
// (1.5 + gamma)(1/rho + 1/sqrt(rho))/a <= 2^76, the total is below 2^-21 c_d, and
// the bounds widen by 2^-20 relative; otherwise the cell is evaluated exactly.
// force = true when no bound is claimed (non-physical or out of FP32 range): the
// caller then evaluates the cell exactly.
template <int PHYS, int NV>
__device__ __forceinline__ void speed_bounds(const double* u, float gam, int ndim, const float* rdx, bool want_rate,
                                             float up[4], float lo[4], bool& force) {
  bool ok = true, fl = false;
  const float rho = f32_of(u[0], ok);
  constexpr int nm = PHYS == PH_EULER ? NV - 2 : 3;
  float m[3] = {0.f, 0.f, 0.f}, B[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < nm; k++) m[k] = f32_of_flush(u[1 + k], ok, fl);
  const float E = f32_of(u[PHYS == PH_EULER ? NV - 1 : 4], ok);
  if (PHYS == PH_MHD) {
#pragma unroll
    for (int k = 0; k < 3; k++) B[k] = f32_of_flush(u[5 + k], ok, fl);
  }
  if (PHYS == PH_MHD && ((dbits(u[8]) >> 52) & 0x7ff) == 0x7ff) ok = false;  // psi not finite
  force = !ok || !(rho > 0.0f) || !(E > 0.0f);
  if (force) return;
  const float ir = __frcp_rn(rho);
  const float v[3] = {m[0] * ir, m[1] * ir, m[2] * ir};
  const float ke2 = fmaf(m[2], v[2], fmaf(m[1], v[1], m[0] * v[0]));
  const float sq[3] = {B[0] * B[0], B[1] * B[1], B[2] * B[2]};
  const float b2 = sq[0] + sq[1] + sq[2];
  const float half = 0.5f * (ke2 + b2);
  const float T = E + half, S = E - half;
  if (!(S > 1.9073486e-6f * T)) { force = true; return; }  // S <= 2^-19 T: too uncertain
  float rel = 7.6293945e-6f * fmaf(T, __frcp_rn(S), 1.0f);  // 2^-17 (T/S + 1)
  const float a2 = gam * (gam - 1.0f) * S * ir;             // gamma p / rho
  if (fl) {
    const float q = (1.5f + gam) * (ir + sqrtf(ir)) / sqrtf(a2);
    if (!(S > 9.765625e-4f * T) || !(q <= 7.5557864e22f)) { force = true; return; }  // 2^-10, 2^76
    rel += 9.5367431640625e-07f;                                                   // 2^-20
  }
  float rate_up = 0.0f, rate_lo = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    if (d >= ndim) { up[d] = 0.0f; lo[d] = 0.0f; continue; }
    float cf;
    if (PHYS == PH_EULER) {
      cf = sqrtf(a2);
    } else {
      const float bd2 = sq[d] * ir;
      const float bt2 = (sq[(d + 1) % 3] + sq[(d + 2) % 3]) * ir;
      const float x = a2 - bd2;
      const float disc = fmaf(x, x, bt2 * (bt2 + 2.0f * (a2 + bd2)));
      cf = sqrtf(0.5f * (a2 + bd2 + bt2 + sqrtf(disc)));
    }
    const float c = fabsf(v[d]) + cf;
    up[d] = c * (1.0f + rel);
    lo[d] = c * (1.0f - rel);
    if (want_rate) {
      rate_up = fmaf(up[d], rdx[d], rate_up);
      rate_lo = fmaf(lo[d], rdx[d], rate_lo);
    }
  }
  up[3] = rate_up * 1.0000153f;  // (1 + 2^-16): rounding of the rate sums and 1/dx
  lo[3] = rate_lo * 0.9999847f;
}

// ------------------------------------------------------ fast flux + LF split
// G^{+-} = F_d +- alpha_d U = 2 F^{+-}: the factor 1/2 of the splitting is
// applied once to the final flux difference (MP5 commutes with scaling by 2
// when its acceptance threshold is scaled by 4).
// Number of per-cell derived quantities the flux needs besides U: MHD v_x, v_y, v_z,
// p_tot = p + B^2/2, v.B; Euler v_1..v_ndim, p.
template <int PHYS, int NV>
struct NumW { static constexpr int value = PHYS == PH_EULER ? NV - 1 : 5; };

// The derived quantities of one cell (the FP64 part of cons -> prim the flux needs).
template <int PHYS, int NV>
__device__ __forceinline__ void prim_w(const double* u, double gm1, double* w) {
  const double ir = frcp(u[0]);
  const double one = ldk(K_ONE), mz = ldk(K_MZ), half = ldk(K_HALF);
  if (PHYS == PH_EULER) {
    constexpr int nm = NV - 2;
    double mv = ldk(K_ZERO);
#pragma unroll
    for (int k = 0; k < nm; k++) { w[k] = rmul(u[1 + k], ir, mz); mv = fma(u[1 + k], w[k], mv); }
    w[nm] = gm1 * fma(-half, mv, u[NV - 1]);
  } else {
    const double v[3] = {rmul(u[1], ir, mz), rmul(u[2], ir, mz), rmul(u[3], ir, mz)};
    const double b2 = fma(u[7], u[7], fma(u[6], u[6], rmul(u[5], u[5], mz)));
    const double mv = fma(u[3], v[2], fma(u[2], v[1], rmul(u[1], v[0], mz)));
    const double p = gm1 * fma(-half, radd(mv, b2, one), u[4]);
    w[0] = v[0]; w[1] = v[1]; w[2] = v[2];
    w[3] = fma(half, b2, p);
    w[4] = fma(v[2], u[7], fma(v[1], u[6], rmul(v[0], u[5], mz)));
  }
}

// Physical flux along D from U and its derived quantities, then the Lax-Friedrichs
// split in doubled form G^{+-} = F +- alpha U (= 2 F^{+-}); psi's flux is c_h^2 B_D.
template <int PHYS, int NV, int D>
__device__ __forceinline__ void split_flux_w(const double* u, const double* w, double alpha, double ch2,
                                             double* gp, double* gm) {
  double f[NV];
  const double one = ldk(K_ONE), mz = ldk(K_MZ);
  if (PHYS == PH_EULER) {
    constexpr int nm = NV - 2;
    const double p = w[nm], vd = w[D];
    f[0] = u[1 + D];
#pragma unroll
    for (int k = 0; k < nm; k++) f[1 + k] = (k == D) ? fma(vd, u[1 + k], p) : rmul(vd, u[1 + k], mz);
    f[NV - 1] = rmul(vd, radd(u[NV - 1], p, one), mz);
  } else {
    const double ptot = w[3], vb = w[4];
    const double vd = w[D], bd = u[5 + D];
    f[0] = u[1 + D];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      f[1 + k] = fma(vd, u[1 + k], rmul(-bd, u[5 + k], mz));
      if (k == D) f[1 + k] = radd(f[1 + k], ptot, one);
      f[5 + k] = (k == D) ? u[8] : fma(vd, u[5 + k], rmul(-bd, w[k], mz));
    }
    f[4] = fma(vd, radd(u[4], ptot, one), rmul(-bd, vb, mz));
    f[8] = rmul(ch2, bd, mz);
  }
#pragma unroll
  for (int v = 0; v < NV; v++) {
    gp[v] = fma(alpha, u[v], f[v]);
    gm[v] = fma(-alpha, u[v], f[v]);
  }
}

// ------------------------------------------------------------- block reductions
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  return x;
}

}  // namespace amrfd
