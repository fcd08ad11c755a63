// amrfd_kernels.cu -- FP64 kernels of the FD-MP5 update (Porth et al. 2014, Sec. 2).
//
//  speeds_kernel   maximal characteristic speed per cell -> per-domain c_max per
//                  direction (Sec. 2.2, "grid-global c_max") and the CFL rate
//                  sum_d c_d/dx_d (Sec. 4.4); exact IEEE operations in the order
//                  of the definition, reduced with integer max on the bit patterns.
//  flux_kernel     one direction's flux difference for a tile of lines:
//                  halo synthesis (periodic / zero-gradient / mirror), the stored
//                  derived quantities, physical flux, Lax-Friedrichs split
//                  G^{+-} = F +- c_max U (Sec. 2.2) into shared memory, then MP5 (or
//                  LIMO3) at every face (Suresh & Huynh 1997, as cited in Sec. 2.2) on
//                  both biases, F^ = R_L(F^+) + R_R(F^-), and -dF^/dx (Sec. 2.1); the
//                  sweeps run in parts, the costliest variable's on a spare warp.
//  combine_kernel  Shu-Osher stage U^(i) = sum a U^(k) + dt b L (Sec. 2.3), GLM psi
//                  damping after the last stage (Sec. 4.2), speeds of U^(i).
//  dt_kernel       dt = CFL / rate per domain, clamped to t_end - t.
//  compact kernels device-side work list of the active blocks (App. C).
#include <cuda_runtime.h>

#include "amrfd_device.cuh"
#include "amrfd_kernels.cuh"

namespace amrfd {

// ----------------------------------------------------------------- utilities
__device__ __forceinline__ void block_coords(const DomDev& dm, int blk, int o[3]) {
  int bx = blk % dm.nb[0];
  int by = (blk / dm.nb[0]) % dm.nb[1];
  int bz = blk / (dm.nb[0] * dm.nb[1]);
  o[0] = bx * dm.be[0];
  o[1] = by * dm.be[1];
  o[2] = bz * dm.be[2];
}

__device__ __forceinline__ DomDev load_dom(const DomDev* p) { return *p; }

// block-wide max of four u64 values; result valid in thread 0
__device__ __forceinline__ void block_max4(unsigned long long v[4], unsigned long long (*red)[32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    unsigned long long x = warp_max_u64(v[q]);
    if (lane == 0) red[q][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      unsigned long long x = lane < nw ? red[q][lane] : 0ull;
      v[q] = warp_max_u64(x);
    }
  }
  __syncthreads();
}

// block-wide max of four non-negative floats, broadcast to every thread
__device__ __forceinline__ void block_max4f_bcast(float v[4], float (*redf)[32], float* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    float x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) redf[q][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      float x = lane < nw ? redf[q][lane] : 0.0f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
      if (lane == 0) out[q] = x;
    }
  }
  __syncthreads();
}

// Exact speeds of one cell folded into the running maxima (IEEE operations in the
// order of the definition); returns false for a non-physical state.
template <int PHYS, int NV>
__device__ __forceinline__ bool exact_speeds(const double* u, double gamma, int ndim, const double* dx, bool want_rate,
                                             unsigned long long mx[4]) {
  Prim w;
  if (!cons2prim_exact<PHYS, NV>(u, gamma, ndim, w)) return false;
  double rate = 0.0;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    if (d < ndim) {
      const double cd = char_speed_exact<PHYS>(w, gamma, d);
      const unsigned long long b = (unsigned long long)dbits(cd);
      mx[d] = b > mx[d] ? b : mx[d];
      if (want_rate) rate = __dadd_rn(rate, __ddiv_rn(cd, dx[d]));
    }
  }
  const unsigned long long br = (unsigned long long)dbits(rate);
  mx[3] = br > mx[3] ? br : mx[3];
  return true;
}

// ------------------------------------------------------------------ speeds
// Exact per-domain maxima in two launches. The bounds launch (exact = 0) evaluates
// FP32 bounds of every active cell's speeds and publishes, per domain, the largest
// lower bound T (an integer max of the FP32 bits), and per item the largest upper bound
// (+inf when a cell carries none). The exact launch (exact = 1) skips the items whose
// upper bounds stay below T, re-evaluates the bounds of the other items' cells and
// computes the exact IEEE speeds only of the cells whose upper bound reaches T, or that
// carry no bound. The maxima are exact: a cell left out lies below T, and T is below the
// speed of the cell that set it. Only the directions d < ndim (and the CFL rate when
// asked for) take part.

template <int PHYS, int NV>
__global__ void __launch_bounds__(256) speeds_kernel(SpeedParams p) {
  __shared__ unsigned long long red[4][32];
  __shared__ float redf[4][32];
  __shared__ float thr[4], thr_up[4];
  const int nitems = p.nitems_dev ? *p.nitems_dev : p.nitems;
  const float gam = (float)p.gamma;
  const bool want_rate = p.want_rate != 0;
  bool on[4];
#pragma unroll
  for (int q = 0; q < 4; q++) on[q] = q < 3 ? q < p.ndim : want_rate;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const CellItem ci = p.items[p.item0 + it];
    AMRFD_GUARD(p.err, cell_item_ok(p.doms, p.ndom, ci), continue)
    const DomDev dm = load_dom(p.doms + ci.dom);
    if (!p.active[dm.block0 + ci.blk]) continue;
    int o[3];
    block_coords(dm, ci.blk, o);
    const float rdx[3] = {(float)(1.0 / dm.dx[0]), (float)(1.0 / dm.dx[1]), (float)(1.0 / dm.dx[2])};
    unsigned* tl = p.tlow + (size_t)ci.dom * 4;
    float* iu = p.item_up ? p.item_up + (size_t)(p.item0 + it) * 4 : nullptr;
    float T[4] = {0.f, 0.f, 0.f, 0.f};
    if (p.exact) {
#pragma unroll
      for (int q = 0; q < 4; q++) T[q] = __uint_as_float(tl[q]);
      if (iu) {  // the same decision in every thread of the block
        bool any = false;
#pragma unroll
        for (int q = 0; q < 4; q++) any |= on[q] && iu[q] >= T[q];
        if (!any) continue;
      }
    }
    unsigned long long mx[4] = {0ull, 0ull, 0ull, 0ull};
    float lom[4] = {0.f, 0.f, 0.f, 0.f};
    float upm[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c = threadIdx.x; c < ci.cnt; c += blockDim.x) {
      const int l = ci.c0 + c;
      const int lx = l % dm.be[0], ly = (l / dm.be[0]) % dm.be[1], lz = l / (dm.be[0] * dm.be[1]);
      const long long idx = dm.off + ((long long)(o[2] + lz) * dm.n[1] + (o[1] + ly)) * dm.n[0] + (o[0] + lx);
      double u[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = p.U[idx + (long long)v * dm.ncell];
      if (p.W) {
        constexpr int NW = NumW<PHYS, NV>::value;
        double w[NW];
        prim_w<PHYS, NV>(u, p.gm1, w);
        const long long wi = dm.woff + (idx - dm.off);
#pragma unroll
        for (int q = 0; q < NW; q++) p.W[wi + (long long)q * dm.ncell] = w[q];
      }
      float up[4], lo[4];
      bool force;
      speed_bounds<PHYS, NV>(u, gam, p.ndim, rdx, want_rate, up, lo, force);
      if (!p.exact) {
        if (!force) {
#pragma unroll
          for (int q = 0; q < 4; q++) {
            lom[q] = fmaxf(lom[q], lo[q]);
            upm[q] = fmaxf(upm[q], up[q]);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; q++) upm[q] = __int_as_float(0x7f800000);  // +inf
        }
        continue;
      }
      bool cand = force;
#pragma unroll
      for (int q = 0; q < 4; q++) cand |= on[q] && up[q] >= T[q];
      if (!cand) continue;
      if (!exact_speeds<PHYS, NV>(u, p.gamma, p.ndim, dm.dx, want_rate, mx)) atomicOr(p.err, kErrNonphysical);
    }
    if (!p.exact) {
      block_max4f_bcast(lom, redf, thr);
      if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (thr[q] > 0.f) atomicMax(tl + q, __float_as_uint(thr[q]));
      if (iu) {
        block_max4f_bcast(upm, redf, thr_up);
        if (threadIdx.x == 0)
#pragma unroll
          for (int q = 0; q < 4; q++) iu[q] = thr_up[q];
      }
      continue;
    }
    block_max4(mx, red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (mx[q]) atomicMax(p.slot + (size_t)ci.dom * 4 + q, mx[q]);
    }
  }
}

// -------------------------------------------------------------------- flux
__device__ __forceinline__ double glm_speed(const unsigned long long* s0, int ndim) {
  double ch = 0.0;
  for (int d = 0; d < ndim; d++) ch = imax(ch, bitsd((long long)s0[d]));
  return ch;
}

// Phase A of a flux item: the tile's G^{+-} (lines x segment + halo) into shared
// memory, cells start, start + stride, ... of the tile.
template <int PHYS, int NV, int D>
__device__ __forceinline__ void flux_phase_a(const FluxParams& p, const DomDev& dm, const FluxItem& it,
                                             const int o[3], double alpha, double ch2, double* sm, int start,
                                             int stride) {
  constexpr int od1 = D == 0 ? 1 : 0;
  constexpr int od2 = D == 2 ? 1 : 2;
  const int W = it.slen + 2 * kGhost;
  const int nl = it.nl;
  const int P = p.P, SS = p.SS;
  const double gm1 = p.gm1;
  for (int c = start; c < nl * W; c += stride) {
    int pl, j;
    if (D == 0) { pl = c / W; j = c - pl * W; }
    else { j = c / nl; pl = c - j * nl; }
    const int line = it.l0 + pl;
    const int a1 = line % dm.be[od1], a2 = line / dm.be[od1];
    int x[3];
    x[od1] = o[od1] + a1;
    x[od2] = o[od2] + a2;
    int g = o[D] + it.s0 + j - kGhost;
    unsigned odd = 0u;  // mirror ghosts: variables negated
    if (g < 0) {
      const int b = dm.bc[D][0];
      odd = dm.asym[D][0];
      g = b == 0 ? g + dm.n[D] : (b == 1 ? 0 : -1 - g);
    } else if (g >= dm.n[D]) {
      const int b = dm.bc[D][1];
      odd = dm.asym[D][1];
      g = b == 0 ? g - dm.n[D] : (b == 1 ? dm.n[D] - 1 : 2 * dm.n[D] - 1 - g);
    }
    x[D] = g;
    AMRFD_GUARD(p.err, g >= 0 && g < dm.n[D] && x[od1] < dm.n[od1] && x[od2] < dm.n[od2] && pl < P && j < SS,
                continue)
    const int nbk = dm.block0 + ((x[2] / dm.be[2]) * dm.nb[1] + x[1] / dm.be[1]) * dm.nb[0] + x[0] / dm.be[0];
    const bool act = p.active[nbk] != 0;
    const double* base = act ? p.Uk : p.Un;
    const long long idx = ((long long)x[2] * dm.n[1] + x[1]) * dm.n[0] + x[0];
    const double* src = base + dm.off + idx;
    constexpr int NW = NumW<PHYS, NV>::value;
    double u[NV], w[NW], gp[NV], gmn[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) u[v] = src[(long long)v * dm.ncell];
    if (odd) {
#pragma unroll
      for (int v = 0; v < NV; v++)
        if ((odd >> v) & 1u) u[v] = dneg(u[v]);
    }
    // derived quantities: stored by the pass that produced U^(k) for active cells;
    // recomputed for passive neighbours (U^n) and mirror images
    if (p.W && act && !odd) {
      const double* ws = p.W + dm.woff + idx;
#pragma unroll
      for (int q = 0; q < NW; q++) w[q] = ws[(long long)q * dm.ncell];
    } else {
      prim_w<PHYS, NV>(u, gm1, w);
    }
    split_flux_w<PHYS, NV, D>(u, w, alpha, ch2, gp, gmn);
#pragma unroll
    for (int v = 0; v < NV; v++) {
      sm[((0 * NV + v) * P + pl) * SS + j] = gp[v];
      sm[((1 * NV + v) * P + pl) * SS + j] = gmn[v];
    }
  }
}

// Recording sweep of one (line, variable): MP5 on both biases at faces k = 3..slen+3 of
// the line's extended index (cell j = k-1 left of face k), then the flux difference
// Fsum_{k-1} - Fsum_k of the segment's cell k-4 stored to out[(k-4) ostr] where wmask has
// its bit (the factor 1/(2 dx) is applied by the stage combination). With
// Fsum_k = G+_{k-1} + G-_k + (Y+_k + Y-_k)/2, the difference is formed from what the sweep
// holds, (S_{k-1} - S_k)/2 - (G+_{k-1} - G+_{k-2}) - (G-_k - G-_{k-1}) with S = Y+ + Y-: no
// subtraction of two fluxes of the size of G, and two shared-memory reads per face (each
// array's newest value; the previous one is kept in a register). Per face and bias it
// records which linear piece the limiter took and the pieces of the two curvature limiters
// it read (mp5_rel2_rec, 3 bits each): tp/tm point at the line's records, face k goes to
// index f0 + k - 3 if below fend (face n of a periodic line, fmod = n, as face 0).
__device__ __forceinline__ void flux_sweep_rec(const double* g, const double* h, int slen, double eps16,
                                               unsigned short* tp, unsigned short* tm, int f0, int fend, int fmod,
                                               double* out, long long ostr, unsigned long long wmask, double one) {
  double Pd1 = rsub(g[1], g[0], one), Pd2 = rsub(g[2], g[1], one), Pd3 = rsub(g[3], g[2], one),
         Pd4 = rsub(g[4], g[3], one);
  double Md2 = rsub(h[2], h[1], one), Md3 = rsub(h[3], h[2], one), Md4 = rsub(h[4], h[3], one),
         Md5 = rsub(h[5], h[4], one);
  double gl = g[4], hl = h[5];  // the last values read, g[k+1] and h[k+2]
  double Sprev = 0.0;
  const int kend = slen + 3;
  for (int k = 3; k <= kend; ++k) {
    int yp, ym;
    const double Yp = mp5_rel2_rec<false>(Pd1, Pd2, Pd3, Pd4, eps16, yp, one);
    const double Ym = mp5_rel2_rec<true>(Md5, Md4, Md3, Md2, eps16, ym, one);
    const int f = f0 + k - 3;
    if (f < fend) {
      const int fi = f >= fmod ? f - fmod : f;
      tp[fi] = (unsigned short)yp;
      tm[fi] = (unsigned short)ym;
    }
    const double S = radd(Yp, Ym, one);
    if (k > 3 && ((wmask >> (k - 4)) & 1ull))
      out[(long long)(k - 4) * ostr] = fma(ldk(K_HALF), rsub(Sprev, S, one), -radd(Pd2, Md3, one));
    Sprev = S;
    if (k < kend) {
      const double gn = g[k + 2], hn = h[k + 3];
      Pd1 = Pd2; Pd2 = Pd3; Pd3 = Pd4; Pd4 = rsub(gn, gl, one); gl = gn;
      Md2 = Md3; Md3 = Md4; Md4 = Md5; Md5 = rsub(hn, hl, one); hl = hn;
    }
  }
}

// Plain MP5 sweep, same fluxes as flux_sweep_rec. The curvature-limited second
// differences serve only faces that fail the acceptance test, so a warp (32 lines of
// one variable) carries them along the line only while some lane keeps failing: after
// a face where one did, it forms them from the current differences (the operands of
// the carried ones) and carries them; after a face where none did, it drops them and
// forms them per face at failing faces only (mp5_rel2_r without CARRY).
// Every lane in `lanes` must call this with the same slen (the face votes pair up).
// Returns the number of faces after which some lane had failed (the same in every lane):
// the warp's limiter work, which phase B uses to balance the variables' sweeps.
__device__ __forceinline__ int flux_sweep_adaptive(const double* g, const double* h, int slen, double eps16,
                                                   double* out, long long ostr, unsigned long long wmask,
                                                   unsigned lanes, double one) {
  int busy = 0;
  double Pd1 = rsub(g[1], g[0], one), Pd2 = rsub(g[2], g[1], one), Pd3 = rsub(g[3], g[2], one),
         Pd4 = rsub(g[4], g[3], one);
  double Md2 = rsub(h[2], h[1], one), Md3 = rsub(h[3], h[2], one), Md4 = rsub(h[4], h[3], one),
         Md5 = rsub(h[5], h[4], one);
  double Pk3 = 0.0, Mk4 = 0.0, PM2 = 0.0, PM3 = 0.0, MM3 = 0.0, MM4 = 0.0;
  bool carry = false;
  double gl = g[4], hl = h[5];  // the last values read, g[k+1] and h[k+2]
  double Sprev = 0.0;
  const int kend = slen + 3;
  for (int k = 3; k <= kend; ++k) {
    // left-biased reconstruction of G^+ centred on cell k-1, right-biased of G^-
    // centred on cell k (mirror image)
    double Yp, Ym;
    bool rp, rm;
    if (carry) {
      Yp = mp5_rel2_r<false, true>(Pd1, Pd2, Pd3, Pd4, PM3, PM2, eps16, rp, one);
      Ym = mp5_rel2_r<true, true>(Md5, Md4, Md3, Md2, MM3, MM4, eps16, rm, one);
    } else {
      Yp = mp5_rel2_r<false, false>(Pd1, Pd2, Pd3, Pd4, 0.0, 0.0, eps16, rp, one);
      Ym = mp5_rel2_r<true, false>(Md5, Md4, Md3, Md2, 0.0, 0.0, eps16, rm, one);
    }
    const double S = radd(Yp, Ym, one);
    if (k > 3 && ((wmask >> (k - 4)) & 1ull))
      out[(long long)(k - 4) * ostr] = fma(ldk(K_HALF), rsub(Sprev, S, one), -radd(Pd2, Md3, one));
    Sprev = S;
    if (k < kend) {
      const bool want = __any_sync(lanes, rp || rm);
      const double gn = g[k + 2], hn = h[k + 3];
      Pd1 = Pd2; Pd2 = Pd3; Pd3 = Pd4; Pd4 = rsub(gn, gl, one); gl = gn;
      Md2 = Md3; Md3 = Md4; Md4 = Md5; Md5 = rsub(hn, hl, one); hl = hn;
      if (want && carry) {
        const double pk = rsub(Pd4, Pd3, one);
        PM2 = PM3;
        PM3 = dm4(Pk3, pk);
        Pk3 = pk;
        const double mk = rsub(Md5, Md4, one);
        MM3 = MM4;
        MM4 = dm4(Mk4, mk);
        Mk4 = mk;
      } else if (want) {
        const double Pk2 = rsub(Pd3, Pd2, one), Mk3 = rsub(Md4, Md3, one);
        Pk3 = rsub(Pd4, Pd3, one);
        Mk4 = rsub(Md5, Md4, one);
        PM2 = dm4(rsub(Pd2, Pd1, one), Pk2);
        PM3 = dm4(Pk2, Pk3);
        MM3 = dm4(rsub(Md3, Md2, one), Mk3);
        MM4 = dm4(Mk3, Mk4);
      }
      carry = want;
      busy += want;
    }
  }
  return busy;
}

// LIMO3 (Cada & Torrilhon 2009) in product form: with a = delta_{i-1/2} and
// b = delta_{i+1/2} (G units), the correction b phi(theta) of u_i + b phi / 2 is
//   unlimited  b phi_3 = (2 b + a) / 3,
//   limited    b phi^_3 = s max(0, min(y3, max(-a'/2, min(2 a', y3, 1.6 |b|))))
// evaluated on a' = s a, y3' = s y3, s = sign(b): multiplying the limiter's terms by
// |b| keeps their order, so no theta = a/b is formed (b = 0 gives 0, the limit). The
// switch eta = (a^2 + b^2) / (4 (r dx)^2) (G = 2 F^{+-}) picks the unlimited value
// inside the asymptotic region, the limited one outside, and blends linearly over
// |eta - 1| < 1e-12.
__device__ __forceinline__ double limo3_y(double a, double b, double s2, long long tlo, long long thi, double esc,
                                          double mz) {
  const double y3 = rmul(fma(ldk(K_TWO), b, a), ldk(K_THIRD), mz);
  const long long bs = abits(s2);  // s2 = a^2 + b^2 >= 0: its bit pattern orders like its value
  if (bs <= tlo) return y3;
  const bool neg = sbit(b) != 0;
  const double ap = neg ? dneg(a) : a;
  const double y3p = neg ? dneg(y3) : y3;
  const double bp = neg ? dneg(b) : b;
  double t = imin(imin(dscale<1>(ap), y3p), rmul(ldk(K_C16), bp, mz));
  t = imax(dscale<-1>(dneg(ap)), t);
  t = imin(y3p, t);
  t = imax(0.0, t);
  const double yl = neg ? dneg(t) : t;
  if (bs >= thi) return yl;
  const double z = fma(s2, esc, -1.0) * 1e12;
  return 0.5 * ((1.0 - z) * y3 + (1.0 + z) * yl);
}

// limo3_y (bit-identical value) that also reports the piece it took, for the discrete
// adjoint: bits 0-2 the limited piece (0 zero, 1 y3, 2 -a/2, 3 2a, 4 1.6 b, each as a
// function of the unsigned a, b), bits 3-4 the mode (0 unlimited, 1 limited, 2 / 3 inside
// the blend band on its unlimited / limited half).
__device__ __forceinline__ double limo3_y_sel(double a, double b, double s2, long long tlo, long long thi,
                                              double esc, int& code, double mz) {
  const double y3 = rmul(fma(ldk(K_TWO), b, a), ldk(K_THIRD), mz);
  const long long bs = abits(s2);
  if (bs <= tlo) { code = 0; return y3; }
  const bool neg = sbit(b) != 0;
  const double ap = neg ? dneg(a) : a;
  const double y3p = neg ? dneg(y3) : y3;
  const double bp = neg ? dneg(b) : b;
  double t;
  int c;
  imin_sel(dscale<1>(ap), 3, y3p, 1, t, c);
  imin_sel(t, c, rmul(ldk(K_C16), bp, mz), 4, t, c);
  imax_sel(dscale<-1>(dneg(ap)), 2, t, c, t, c);
  imin_sel(y3p, 1, t, c, t, c);
  imax_sel(0.0, 0, t, c, t, c);
  const double yl = neg ? dneg(t) : t;
  if (bs >= thi) { code = c | (1 << 3); return yl; }
  const double z = fma(s2, esc, -1.0) * 1e12;
  code = c | ((z < 0.0 ? 2 : 3) << 3);
  return 0.5 * ((1.0 - z) * y3 + (1.0 + z) * yl);
}

// LIMO3 sweep of one (line, variable): faces k = 3..slen+3 as in flux_sweep_rec; G^+ from
// cells k-2..k (centre k-1), G^- mirrored from cells k+1..k-1 (centre k). The squares of
// the differences are carried along the line (each enters two faces' switch), and the
// switch compares a^2 + b^2 with (1 -+ 1e-12)/esc.
__device__ __forceinline__ void limo3_sweep(const double* g, const double* h, int slen, double esc, double* out,
                                            long long ostr, unsigned long long wmask) {
  const long long tlo = __double_as_longlong((1.0 - 1e-12) / esc), thi = __double_as_longlong((1.0 + 1e-12) / esc);
  const double one = ldk(K_ONE), mz = ldk(K_MZ);
  double Pa = rsub(g[2], g[1], one), Pb = rsub(g[3], g[2], one);  // delta_{i-1/2}, delta_{i+1/2} of G^+ at face 3
  double Mb = rsub(h[3], h[2], one), Ma = rsub(h[4], h[3], one);  // mirrored: -delta_{i+1/2}, -delta_{i-1/2} of G^-
  double Pa2 = rmul(Pa, Pa, mz), Pb2 = rmul(Pb, Pb, mz), Ma2 = rmul(Ma, Ma, mz), Mb2 = rmul(Mb, Mb, mz);
  double gl = g[3], hl = h[4];  // the last values read, g[k] and h[k+1]
  double Sprev = 0.0;
  const int kend = slen + 3;
  for (int k = 3; k <= kend; ++k) {
    const double Yp = limo3_y(Pa, Pb, radd(Pa2, Pb2, one), tlo, thi, esc, mz);
    const double Ym = limo3_y(Ma, Mb, radd(Ma2, Mb2, one), tlo, thi, esc, mz);
    const double S = rsub(Yp, Ym, one);
    if (k > 3 && ((wmask >> (k - 4)) & 1ull))
      out[(long long)(k - 4) * ostr] = fma(ldk(K_HALF), rsub(Sprev, S, one), -radd(Pa, Mb, one));
    Sprev = S;
    if (k < kend) {
      const double gn = g[k + 1], hn = h[k + 2];
      Pa = Pb; Pa2 = Pb2; Pb = rsub(gn, gl, one); Pb2 = rmul(Pb, Pb, mz); gl = gn;
      Mb = Ma; Mb2 = Ma2; Ma = rsub(hn, hl, one); Ma2 = rmul(Ma, Ma, mz); hl = hn;
    }
  }
}

// limo3_sweep that also records, per face and bias, the piece LIMO3 took (limo3_y_sel),
// faces f0 + k - 3 below fend as flux_sweep_rec records them.
__device__ __forceinline__ void limo3_sweep_rec(const double* g, const double* h, int slen, double esc,
                                                unsigned short* tp, unsigned short* tm, int f0, int fend, int fmod,
                                                double* out, long long ostr, unsigned long long wmask) {
  const long long tlo = __double_as_longlong((1.0 - 1e-12) / esc), thi = __double_as_longlong((1.0 + 1e-12) / esc);
  const double one = ldk(K_ONE), mz = ldk(K_MZ);
  double Pa = rsub(g[2], g[1], one), Pb = rsub(g[3], g[2], one);
  double Mb = rsub(h[3], h[2], one), Ma = rsub(h[4], h[3], one);
  double Pa2 = rmul(Pa, Pa, mz), Pb2 = rmul(Pb, Pb, mz), Ma2 = rmul(Ma, Ma, mz), Mb2 = rmul(Mb, Mb, mz);
  double gl = g[3], hl = h[4];  // the last values read, g[k] and h[k+1]
  double Sprev = 0.0;
  const int kend = slen + 3;
  for (int k = 3; k <= kend; ++k) {
    int cp, cm;
    const double Yp = limo3_y_sel(Pa, Pb, radd(Pa2, Pb2, one), tlo, thi, esc, cp, mz);
    const double Ym = limo3_y_sel(Ma, Mb, radd(Ma2, Mb2, one), tlo, thi, esc, cm, mz);
    const int f = f0 + k - 3;
    if (f < fend) {
      const int fi = f >= fmod ? f - fmod : f;  // face n of a periodic line is face 0
      tp[fi] = (unsigned short)cp;
      tm[fi] = (unsigned short)cm;
    }
    const double S = rsub(Yp, Ym, one);
    if (k > 3 && ((wmask >> (k - 4)) & 1ull))
      out[(long long)(k - 4) * ostr] = fma(ldk(K_HALF), rsub(Sprev, S, one), -radd(Pa, Mb, one));
    Sprev = S;
    if (k < kend) {
      const double gn = g[k + 1], hn = h[k + 2];
      Pa = Pb; Pa2 = Pb2; Pb = rsub(gn, gl, one); Pb2 = rmul(Pb, Pb, mz); gl = gn;
      Mb = Ma; Mb2 = Ma2; Ma = rsub(hn, hl, one); Ma2 = rmul(Ma, Ma, mz); hl = hn;
    }
  }
}

// Splitting speed of an item's direction (raised to c_h with GLM) and c_h^2.
template <int D>
__device__ __forceinline__ double item_alpha(const FluxParams& p, const FluxItem& it, double& ch2) {
  const unsigned long long* sk = p.araw + (size_t)it.dom * 4;
  const unsigned long long* s0 = p.araw0 + (size_t)it.dom * 4;
  const double ch = p.glm ? glm_speed(s0, p.ndim) : 0.0;
  ch2 = ch * ch;
  return imax(bitsd((long long)sk[D]), ch);
}

// Whether any / every block the item's segment runs through is active.
__device__ __forceinline__ bool item_live(const FluxParams& p, const FluxItem& item, bool& all_live) {
  const DomDev& dm = p.doms[item.dom];
  const int d = item.d;
  const int bidx[3] = {item.blk % dm.nb[0], (item.blk / dm.nb[0]) % dm.nb[1], item.blk / (dm.nb[0] * dm.nb[1])};
  const int stride = d == 0 ? 1 : (d == 1 ? dm.nb[0] : dm.nb[0] * dm.nb[1]);
  const int c0 = bidx[d] * dm.be[d] + item.s0;
  const int b0 = c0 / dm.be[d], b1 = (c0 + item.slen - 1) / dm.be[d];
  const int g0 = dm.block0 + item.blk + (b0 - bidx[d]) * stride;
  bool live = false;
  all_live = true;
  for (int b = b0; b <= b1; b++) {
    const bool a = p.active[g0 + (b - b0) * stride] != 0;
    live |= a;
    all_live &= a;
  }
  return live;
}

// Parts of a segment's sweep: a segment of 32 cells or more is swept in np equal parts
// of at least 16 cells (np the largest divisor of slen up to slen/16), one thread per
// (variable, part, line); each part recomputes the face at its left end, as a 16-cell
// segment does. Longer segments then cost less halo work in phase A (6 cells per
// segment) without leaving phase-B threads idle. Equal parts keep every sweep of an
// item equally long, which the adaptive sweep's per-face votes need.
constexpr int kPartMin = 16;
__device__ __forceinline__ int sweep_parts(int slen) {
  int np = slen / kPartMin;
  while (np > 1 && slen % np) np--;
  return np > 1 ? np : 1;
}

// The variable whose MP5 sweeps cost clearly most, from the CTA's decaying per-variable
// counts of limiter faces (cost[v]), or -1: its count must exceed the runner-up's by an
// eighth (and a few faces).
template <int NV>
__device__ __forceinline__ int hot_variable(const unsigned* cost) {
  int h = -1;
  unsigned m1 = 0u, m2 = 0u;
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const unsigned c = cost[v];
    if (c > m1) { m2 = m1; m1 = c; h = v; }
    else if (c > m2) m2 = c;
  }
  return m1 > m2 + (m2 >> 3) + 4u ? h : -1;
}

// Phase B of a flux item: one thread per (variable, part, line) sweeps the part's faces
// and stores L_D of its cells (MODE 0: MP5; 1: MP5 recording the limiter pieces;
// 2: LIMO3; 3: LIMO3 recording its pieces). The loop runs warp by warp: every lane of a
// warp takes the same number of trips, so that the adaptive sweep's per-face votes see
// exactly the lanes holding work, all of them sweeping parts of the same length.
// Balance (MODE 0): a variable whose faces fail the MP5 acceptance test far more often
// than the others' (noise in one variable, a contact discontinuity) makes its warps the
// slowest, and the others wait for them at the CTA barrier. The costliest variable `hot`
// (hot_variable, from the CTA's earlier items) is then swept in twice as many parts of
// half the length, on twice the warps, when every variable's tasks fill whole warps and
// the CTA has threads for the extra tasks. A face's value does not depend on the part
// that computes it, so the results are the same bit for bit. Each warp adds its limiter
// face count to cost_new[v].
template <int PHYS, int NV, int D, int MODE>
__device__ __forceinline__ void flux_phase_b(const FluxParams& p, const DomDev& dm, const FluxItem& it,
                                             const int o[3], bool all_live, const double* sm,
                                             const unsigned* cost, unsigned* cost_new) {
  constexpr bool REC = MODE == 1 || MODE == 3;
  const int nl = it.nl, slen = it.slen;
  const int np = sweep_parts(slen);
  // MP5 acceptance (f_or - f_i)(f_or - f_mp) <= 1e-10 for F^{+-}; G = 2 F^{+-} and the
  // doubled relative values of mp5_rel2_r scale the product by 16 (exactly)
  const double eps16 = 16.0 * 1e-10;
  constexpr int od1 = D == 0 ? 1 : 0;
  constexpr int od2 = D == 2 ? 1 : 2;
  const int f0 = o[D] + it.s0;
  const long long nlines = (long long)dm.n[od1] * dm.n[od2];
  const int bstride = D == 0 ? 1 : (D == 1 ? dm.nb[0] : dm.nb[0] * dm.nb[1]);
  const int bo = it.blk - (o[D] / dm.be[D]) * bstride;  // block index with coordinate D = 0
  // faces the segment's sweeps record (REC): those it owns, f0 .. f0 + slen - 1, and the
  // face after it where no segment owning that face runs: at an outflow or mirror end of
  // the line, or before a passive block (whose segments the forward pass skips; the
  // adjoint reads the face there). On a periodic line face n is face 0.
  int fend = f0 + slen;
  {
    const bool at_end = f0 + slen == dm.n[D];
    if (at_end && dm.bc[D][1] != 0) fend++;
    else if (REC && !p.active[dm.block0 + bo + ((at_end ? 0 : f0 + slen) / dm.be[D]) * bstride]) fend++;
  }
  const int fmod = dm.bc[D][1] == 0 ? dm.n[D] : dm.n[D] + 1;
  // cells of the segment inside active blocks (a segment through several blocks may
  // cross a passive one; every line of the item crosses the same blocks)
  unsigned long long wmask = slen >= 64 ? ~0ull : ((1ull << slen) - 1ull);
  if (!all_live) {
    for (int j = 0; j < slen; j++)
      if (!p.active[dm.block0 + bo + ((o[D] + it.s0 + j) / dm.be[D]) * bstride]) wmask &= ~(1ull << j);
  }
  const long long ostr = D == 0 ? 1 : (D == 1 ? (long long)dm.n[0] : (long long)dm.n[0] * dm.n[1]);
  double* Ld = p.L[D] + dm.off;
  const int nh = nl * np;  // tasks per variable
  int hot = -1;
  if (MODE == 0 && nh % 32 == 0 && (slen / np) % 2 == 0 && slen / np >= 2 * 8 && nh * (NV + 1) <= (int)blockDim.x)
    hot = hot_variable<NV>(cost);
  const int total = nh * NV + (hot >= 0 ? nh : 0);
  const int lane = threadIdx.x & 31;
  const double one = ldk(K_ONE);
  for (int t0 = threadIdx.x - lane; t0 < total; t0 += blockDim.x) {
    const int t = t0 + lane;
    const bool valid = t < total;
    int plen = slen / np;
    int pl = 0, v = 0, q = 0;
    if (valid) {  // a warp holds consecutive parts and lines of one variable
      if (hot < 0) {
        pl = t % nl;
        const int r = t / nl;
        q = r % np;
        v = r / np;
      } else if (t < 2 * nh) {  // the hot variable first: 2 np parts of plen / 2 cells
        v = hot;
        plen >>= 1;
        pl = t % nl;
        q = t / nl;
      } else {
        const int u = t - 2 * nh, vi = u / nh, r = u - vi * nh;
        v = vi < hot ? vi : vi + 1;
        pl = r % nl;
        q = r / nl;
      }
    }
    const int p0 = q * plen;
    const unsigned vm = __ballot_sync(0xffffffffu, valid);
    if (!valid) continue;
    const double* g = sm + ((0 * NV + v) * p.P + pl) * p.SS + p0;
    const double* h = sm + ((1 * NV + v) * p.P + pl) * p.SS + p0;
    const int line = it.l0 + pl;
    const int a1 = line % dm.be[od1], a2 = line / dm.be[od1];
    int x[3];
    x[od1] = o[od1] + a1;
    x[od2] = o[od2] + a2;
    x[D] = o[D] + it.s0 + p0;
    double* out = Ld + (long long)v * dm.ncell + ((long long)x[2] * dm.n[1] + x[1]) * dm.n[0] + x[0];
    const unsigned long long pmask = (wmask >> p0) & (plen >= 64 ? ~0ull : ((1ull << plen) - 1ull));
    if constexpr (MODE == 2) {
      const double rdx = p.limo3_r * dm.dx[D];
      limo3_sweep(g, h, plen, 0.25 / (rdx * rdx), out, ostr, pmask);
    } else if constexpr (REC) {
      const long long ld = (long long)(o[od2] + a2) * dm.n[od1] + (o[od1] + a1);
      unsigned short* tp = p.tape + dm.tape_off[D] + ((long long)(v * 2 + 0) * nlines + ld) * (dm.n[D] + 1);
      unsigned short* tm = p.tape + dm.tape_off[D] + ((long long)(v * 2 + 1) * nlines + ld) * (dm.n[D] + 1);
      // a part records the faces it owns: its left face and interior faces; the
      // segment's last part also the faces the segment owns at its right end
      const int fe = q == np - 1 ? fend : f0 + p0 + plen;
      if constexpr (MODE == 3) {
        const double rdx = p.limo3_r * dm.dx[D];
        limo3_sweep_rec(g, h, plen, 0.25 / (rdx * rdx), tp, tm, f0 + p0, fe, fmod, out, ostr, pmask);
      } else {
        flux_sweep_rec(g, h, plen, eps16, tp, tm, f0 + p0, fe, fmod, out, ostr, pmask, one);
      }
    } else {
      const int busy = flux_sweep_adaptive(g, h, plen, eps16, out, ostr, pmask, vm, one);
      if (lane == __ffs(vm) - 1 && busy) atomicAdd(cost_new + v, (unsigned)busy);
    }
  }
}

// One flux item by the whole CTA: phase A, barrier, phase B, barrier.
// cost[0..NV) holds the CTA's decaying per-variable limiter counts, cost[16..16+NV) this
// item's; every count of the previous item was added before the barrier that ended it.
template <int PHYS, int NV, int D, int MODE>
__device__ __forceinline__ void flux_item(const FluxParams& p, const FluxItem& it, double* sm, bool all_live,
                                          unsigned* cost) {
  if (threadIdx.x < NV) {
    const unsigned c = cost[threadIdx.x];
    cost[threadIdx.x] = c - (c >> 2) + cost[16 + threadIdx.x];
    cost[16 + threadIdx.x] = 0u;
  }
  const DomDev dm = load_dom(p.doms + it.dom);
  int o[3];
  block_coords(dm, it.blk, o);
  double ch2;
  const double alpha = item_alpha<D>(p, it, ch2);
  flux_phase_a<PHYS, NV, D>(p, dm, it, o, alpha, ch2, sm, threadIdx.x, blockDim.x);
  __syncthreads();
  flux_phase_b<PHYS, NV, D, MODE>(p, dm, it, o, all_live, sm, cost, cost + 16);
  __syncthreads();
}

template <int PHYS, int NV, int MODE>
__global__ void __launch_bounds__(kFluxMaxThreads, 2) flux_kernel(FluxParams p) {
  extern __shared__ double sm[];
  __shared__ int s_it;
  __shared__ unsigned s_cost[32];
  if (threadIdx.x < 16) {  // each slot pair is read (flux_item) by the thread that zeroes it
    s_cost[threadIdx.x] = 0u;
    s_cost[16 + threadIdx.x] = 0u;
  }
  const int nitems = p.nitems_dev ? *p.nitems_dev : p.nitems;
  int it;
  if (p.counter) {
    if (threadIdx.x == 0) s_it = atomicAdd(p.counter, 1);
    __syncthreads();
    it = s_it;
    __syncthreads();
  } else {
    it = blockIdx.x;
  }
  constexpr int maxd = PHYS == PH_EULER ? NV - 2 : 3;
  while (it < nitems) {
    const FluxItem item = p.items[p.item0 + it];
    bool all_live = false;
    bool live = true;
    AMRFD_GUARD(p.err, flux_item_ok(p.doms, p.ndom, p.ndim, p.P, p.SS, item), live = false)
    live = live && item_live(p, item, all_live);
    if (live && item.d == 0) flux_item<PHYS, NV, 0, MODE>(p, item, sm, all_live, s_cost);
    if constexpr (maxd > 1) { if (live && item.d == 1) flux_item<PHYS, NV, (maxd > 1 ? 1 : 0), MODE>(p, item, sm, all_live, s_cost); }
    if constexpr (maxd > 2) { if (live && item.d == 2) flux_item<PHYS, NV, (maxd > 2 ? 2 : 0), MODE>(p, item, sm, all_live, s_cost); }
    if (p.counter) {
      if (threadIdx.x == 0) s_it = atomicAdd(p.counter, 1);
      __syncthreads();
      it = s_it;
      __syncthreads();
    } else {
      it += gridDim.x;
    }
  }
}

// ----------------------------------------------------------------- combine
// The derived quantities and FP32 speed bounds of one new state u (cell at idx).
template <int PHYS, int NV>
__device__ __forceinline__ void combine_tail(const CombParams& p, const DomDev& dm, long long idx, const double* u,
                                             float gam, float lom[4], float upm[4]) {
  const float rdx[3] = {0.f, 0.f, 0.f};
  if (p.W) {
    constexpr int NW = NumW<PHYS, NV>::value;
    double w[NW];
    prim_w<PHYS, NV>(u, p.gm1, w);
    const long long wi = dm.woff + (idx - dm.off);
#pragma unroll
    for (int q = 0; q < NW; q++) p.W[wi + (long long)q * dm.ncell] = w[q];
  }
  if (p.tlow_out) {
    float up[4], lo[4];
    bool force;
    speed_bounds<PHYS, NV>(u, gam, p.ndim, rdx, false, up, lo, force);
    if (!force) {
#pragma unroll
      for (int q = 0; q < 3; q++) {
        lom[q] = fmaxf(lom[q], lo[q]);
        upm[q] = fmaxf(upm[q], up[q]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 3; q++) upm[q] = __int_as_float(0x7f800000);  // +inf
    }
  }
}

// The cells of one item. Every load of a cell is issued before its stores (the output
// may be the U^n buffer, so loads cannot move past a store); A0ONE skips the product
// with a first coefficient of 1. Per variable the operations and their order are
// a_0 U^(k_0), then a_t U^(k_t) and w_d L_d by FMA, then the psi damping.
template <int PHYS, int NV, bool A0ONE>
__device__ __forceinline__ void combine_cells(const CombParams& p, const DomDev& dm, const CellItem& ci,
                                              const int o[3], double w0, double w1, double w2, double fac,
                                              float gam, float lom[4], float upm[4]) {
  const long long nc = dm.ncell;
  for (int c = threadIdx.x; c < ci.cnt; c += blockDim.x) {
    const int l = ci.c0 + c;
    const int lx = l % dm.be[0], ly = (l / dm.be[0]) % dm.be[1], lz = l / (dm.be[0] * dm.be[1]);
    const long long idx = dm.off + ((long long)(o[2] + lz) * dm.n[1] + (o[1] + ly)) * dm.n[0] + (o[0] + lx);
    double u[NV];
    {
      const double* b0 = p.buf[p.co.k[0]] + idx;
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = A0ONE ? b0[v * nc] : p.co.a[0] * b0[v * nc];
    }
    for (int t = 1; t < p.co.nterm; t++) {
      const double* bt = p.buf[p.co.k[t]] + idx;
      const double at = p.co.a[t];
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = fma(at, bt[v * nc], u[v]);
    }
    {
      const double* L0 = p.L[0] + idx;
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = fma(w0, L0[v * nc], u[v]);
    }
    if (p.ndim > 1) {
      const double* L1 = p.L[1] + idx;
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = fma(w1, L1[v * nc], u[v]);
    }
    if (p.ndim > 2) {
      const double* L2 = p.L[2] + idx;
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = fma(w2, L2[v * nc], u[v]);
    }
    if constexpr (PHYS == PH_MHD) u[NV - 1] *= fac;  // psi
#pragma unroll
    for (int v = 0; v < NV; v++) p.out[idx + v * nc] = u[v];
    combine_tail<PHYS, NV>(p, dm, idx, u, gam, lom, upm);
  }
}

// combine_cells for two neighbouring cells along x per thread, read and written with
// 16-byte (double2) accesses; the same operations in the same order on each cell. The
// caller checks that every pair starts 16-byte aligned.
template <int PHYS, int NV, bool A0ONE>
__device__ __forceinline__ void combine_pairs(const CombParams& p, const DomDev& dm, const CellItem& ci,
                                              const int o[3], double w0, double w1, double w2, double fac,
                                              float gam, float lom[4], float upm[4]) {
  const long long nc = dm.ncell;
  for (int c = threadIdx.x; c < ci.cnt / 2; c += blockDim.x) {
    const int l = ci.c0 + 2 * c;
    const int lx = l % dm.be[0], ly = (l / dm.be[0]) % dm.be[1], lz = l / (dm.be[0] * dm.be[1]);
    const long long idx = dm.off + ((long long)(o[2] + lz) * dm.n[1] + (o[1] + ly)) * dm.n[0] + (o[0] + lx);
    double ua[NV], ub[NV];
    {
      const double* b0 = p.buf[p.co.k[0]] + idx;
#pragma unroll
      for (int v = 0; v < NV; v++) {
        const double2 x = *reinterpret_cast<const double2*>(b0 + v * nc);
        ua[v] = A0ONE ? x.x : p.co.a[0] * x.x;
        ub[v] = A0ONE ? x.y : p.co.a[0] * x.y;
      }
    }
    for (int t = 1; t < p.co.nterm; t++) {
      const double* bt = p.buf[p.co.k[t]] + idx;
      const double at = p.co.a[t];
#pragma unroll
      for (int v = 0; v < NV; v++) {
        const double2 x = *reinterpret_cast<const double2*>(bt + v * nc);
        ua[v] = fma(at, x.x, ua[v]);
        ub[v] = fma(at, x.y, ub[v]);
      }
    }
    for (int d = 0; d < p.ndim; d++) {
      const double* Ld = p.L[d] + idx;
      const double wd = d == 0 ? w0 : (d == 1 ? w1 : w2);
#pragma unroll
      for (int v = 0; v < NV; v++) {
        const double2 x = *reinterpret_cast<const double2*>(Ld + v * nc);
        ua[v] = fma(wd, x.x, ua[v]);
        ub[v] = fma(wd, x.y, ub[v]);
      }
    }
    if constexpr (PHYS == PH_MHD) {
      ua[NV - 1] *= fac;  // psi
      ub[NV - 1] *= fac;
    }
#pragma unroll
    for (int v = 0; v < NV; v++) *reinterpret_cast<double2*>(p.out + idx + v * nc) = make_double2(ua[v], ub[v]);
    for (int half = 0; half < 2; half++) combine_tail<PHYS, NV>(p, dm, idx + half, half ? ub : ua, gam, lom, upm);
  }
}

template <int PHYS, int NV>
__global__ void __launch_bounds__(256) combine_kernel(CombParams p) {
  __shared__ float redf[4][32];
  __shared__ float thr[4], thr_up[4];
  __shared__ double s_fac;
  const int nitems = p.nitems_dev ? *p.nitems_dev : p.nitems;
  const float gam = (float)p.gamma;
  const bool a0_one = p.co.a[0] == 1.0;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const CellItem ci = p.items[p.item0 + it];
    AMRFD_GUARD(p.err, cell_item_ok(p.doms, p.ndom, ci), continue)
    const DomDev dm = load_dom(p.doms + ci.dom);
    if (!p.active[dm.block0 + ci.blk]) continue;
    int o[3];
    block_coords(dm, ci.blk, o);
    const double dt = p.dt[ci.dom];
    const double dtb = dt * p.co.b;
    // L = sum_d (Fsum_{i-1/2} - Fsum_{i+1/2}) / (2 dx_d), Fsum in units of 2 F^
    const double w0 = dtb * (0.5 / dm.dx[0]);
    const double w1 = p.ndim > 1 ? dtb * (0.5 / dm.dx[1]) : 0.0;
    const double w2 = p.ndim > 2 ? dtb * (0.5 / dm.dx[2]) : 0.0;
    const bool damp = PHYS == PH_MHD && p.final_stage && p.glm_cr > 0.0;
    if (damp) {
      if (threadIdx.x == 0) {
        const double ch = glm_speed(p.araw0 + (size_t)ci.dom * 4, p.ndim);
        s_fac = exp(-dt * ch / p.glm_cr);
      }
      __syncthreads();
    }
    const double fac = damp ? s_fac : 1.0;
    float lom[4] = {0.f, 0.f, 0.f, 0.f};
    float upm[4] = {0.f, 0.f, 0.f, 0.f};
    // pairs along x when every pair starts 16-byte aligned: buffers aligned (host), an even
    // x extent and block edge, an even domain offset and item start and count
    const bool pair = p.pairs && !((dm.n[0] | dm.be[0] | ci.c0 | ci.cnt) & 1) && !(dm.off & 1);
    if (pair) {
      if (a0_one) combine_pairs<PHYS, NV, true>(p, dm, ci, o, w0, w1, w2, fac, gam, lom, upm);
      else combine_pairs<PHYS, NV, false>(p, dm, ci, o, w0, w1, w2, fac, gam, lom, upm);
    } else {
      if (a0_one) combine_cells<PHYS, NV, true>(p, dm, ci, o, w0, w1, w2, fac, gam, lom, upm);
      else combine_cells<PHYS, NV, false>(p, dm, ci, o, w0, w1, w2, fac, gam, lom, upm);
    }
    if (p.tlow_out) {
      block_max4f_bcast(lom, redf, thr);
      if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 3; q++)
          if (thr[q] > 0.f) atomicMax(p.tlow_out + (size_t)ci.dom * 4 + q, __float_as_uint(thr[q]));
      if (p.item_up) {
        block_max4f_bcast(upm, redf, thr_up);
        if (threadIdx.x == 0)
#pragma unroll
          for (int q = 0; q < 4; q++) p.item_up[(size_t)(p.item0 + it) * 4 + q] = thr_up[q];
      }
    } else if (damp) {
      __syncthreads();  // s_fac is rewritten by the next item
    }
  }
}

// --------------------------------------------------------------------- dt
__global__ void __launch_bounds__(1024) dt_kernel(DtParams p) {
  __shared__ long long red[32];
  long long best = 0x7fffffffffffffffLL;  // okey of the minimum over this thread's domains
  for (int dmi = threadIdx.x; dmi < p.ndom; dmi += blockDim.x) {
    const DomDev& dm = p.doms[dmi];
    const unsigned long long* s = p.slot + (size_t)dmi * 4;
    double rate;
    if (p.glm) {
      double ch = 0.0;
      for (int d = 0; d < p.ndim; d++) ch = imax(ch, bitsd((long long)s[d]));
      rate = 0.0;
      for (int d = 0; d < p.ndim; d++) rate = __dadd_rn(rate, __ddiv_rn(ch, dm.dx[d]));
    } else {
      rate = bitsd((long long)s[3]);
    }
    double dt = rate > 0.0 ? __ddiv_rn(p.cfl, rate) : __longlong_as_double(0x7ff0000000000000LL);
    const double rem = __dsub_rn(p.t_end, p.t);
    dt = imin(dt, rem);
    p.dt_out[dmi] = dt;
    const long long k = okey(dt);
    best = k < best ? k : best;
  }
  if (!p.global_min) return;
  for (int o = 16; o > 0; o >>= 1) {
    long long y = __shfl_xor_sync(0xffffffffu, best, o);
    best = y < best ? y : best;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    long long x = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0x7fffffffffffffffLL;
    for (int o = 16; o > 0; o >>= 1) {
      long long y = __shfl_xor_sync(0xffffffffu, x, o);
      x = y < x ? y : x;
    }
    if (threadIdx.x == 0) red[0] = x;
  }
  __syncthreads();
  const long long kb = red[0];
  const double dmin = bitsd(kb ^ ((kb >> 63) & 0x7fffffffffffffffLL));
  for (int dmi = threadIdx.x; dmi < p.ndom; dmi += blockDim.x) p.dt_out[dmi] = dmin;
}

// ------------------------------------------------------------- compaction
__device__ __forceinline__ bool group_live(const CompactParams& p, int i) {
  const int o = p.list.owner[i], st = p.list.stride[i], sp = p.list.span[i];
  bool live = false;
  for (int m = 0; m < sp; m++) live |= p.active[o + m * st] != 0;
  return live;
}

__global__ void __launch_bounds__(1024) compact_scan_kernel(CompactParams p) {
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < p.list.ngroups; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int f = (i < p.list.ngroups && group_live(p, i)) ? p.list.cnt[i] : 0;
    int fs = f;
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(0xffffffffu, fs, o);
      if (lane >= o) fs += a;
    }
    if (lane == 31) wsum[wid] = fs;
    __syncthreads();
    if (wid == 0) {
      const int nw = blockDim.x >> 5;
      int a = lane < nw ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, a, o);
        if (lane >= o) a += x;
      }
      if (lane < nw) wsum[lane] = a;
    }
    __syncthreads();
    const int fo = carry + (wid ? wsum[wid - 1] : 0) + fs - f;
    if (i < p.list.ngroups) p.list.dst[i] = f ? fo : -1;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = fo + f;
    __syncthreads();
  }
  if (threadIdx.x == 0) *p.list.count = carry;
}

__global__ void __launch_bounds__(256) compact_copy_kernel(CompactParams p) {
  const int w = p.list.item_bytes / 4;
  const unsigned* in = (const unsigned*)p.list.in;
  unsigned* out = (unsigned*)p.list.out;
  for (int i = blockIdx.x; i < p.list.ngroups; i += gridDim.x) {
    const int d = p.list.dst[i];
    if (d < 0) continue;
    const int b = p.list.beg[i], c = p.list.cnt[i];
    for (int t = threadIdx.x; t < c * w; t += blockDim.x) out[(size_t)d * w + t] = in[(size_t)b * w + t];
  }
}

// ------------------------------------------------------------- dispatch
#define AMRFD_DISPATCH(physics, nv, CALL)                                   \
  do {                                                                      \
    if ((physics) == PH_MHD && (nv) == 9) { CALL(PH_MHD, 9); }              \
    else if ((physics) == PH_EULER && (nv) == 3) { CALL(PH_EULER, 3); }     \
    else if ((physics) == PH_EULER && (nv) == 4) { CALL(PH_EULER, 4); }     \
    else if ((physics) == PH_EULER && (nv) == 5) { CALL(PH_EULER, 5); }     \
    else return cudaErrorInvalidValue;                                      \
  } while (0)

cudaError_t launch_speeds(int physics, int nv, const SpeedParams& p, int grid, int block, cudaStream_t s) {
#define CALL(PH, NVV) speeds_kernel<PH, NVV><<<grid, block, 0, s>>>(p)
  AMRFD_DISPATCH(physics, nv, CALL);
#undef CALL
  return cudaGetLastError();
}

cudaError_t launch_flux(int physics, int nv, const FluxParams& p, int grid, int block, size_t smem, cudaStream_t s) {
#define CALL(PH, NVV)                                                                \
  if (p.tape && p.limo3) flux_kernel<PH, NVV, 3><<<grid, block, smem, s>>>(p);      \
  else if (p.tape) flux_kernel<PH, NVV, 1><<<grid, block, smem, s>>>(p);            \
  else if (p.limo3) flux_kernel<PH, NVV, 2><<<grid, block, smem, s>>>(p);           \
  else flux_kernel<PH, NVV, 0><<<grid, block, smem, s>>>(p)
  AMRFD_DISPATCH(physics, nv, CALL);
#undef CALL
  return cudaGetLastError();
}

cudaError_t flux_set_smem(int physics, int nv, size_t smem) {
#define CALL(PH, NVV)                                                                                     \
  do {                                                                                                     \
    cudaError_t e = cudaFuncSetAttribute(flux_kernel<PH, NVV, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                                                       \
    if (e != cudaSuccess) return e;                                                                        \
    return cudaFuncSetAttribute(flux_kernel<PH, NVV, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
  } while (0)
  AMRFD_DISPATCH(physics, nv, CALL);
#undef CALL
  return cudaSuccess;
}

cudaError_t flux_rec_set_smem(int physics, int nv, size_t smem) {
#define CALL(PH, NVV)                                                                                     \
  do {                                                                                                     \
    cudaError_t e = cudaFuncSetAttribute(flux_kernel<PH, NVV, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                                                       \
    if (e != cudaSuccess) return e;                                                                        \
    return cudaFuncSetAttribute(flux_kernel<PH, NVV, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
  } while (0)
  AMRFD_DISPATCH(physics, nv, CALL);
#undef CALL
  return cudaSuccess;
}

cudaError_t flux_occupancy(int physics, int nv, int limo3, int block, size_t smem, int* per_sm) {
#define CALL(PH, NVV)                                                                                        \
  return limo3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, flux_kernel<PH, NVV, 2>, block, smem) \
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, flux_kernel<PH, NVV, 0>, block, smem)
  AMRFD_DISPATCH(physics, nv, CALL);
#undef CALL
  return cudaSuccess;
}

cudaError_t launch_combine(int physics, int nv, const CombParams& p, int grid, int block, cudaStream_t s) {
#define CALL(PH, NVV) combine_kernel<PH, NVV><<<grid, block, 0, s>>>(p)
  AMRFD_DISPATCH(physics, nv, CALL);
#undef CALL
  return cudaGetLastError();
}

// One round of App. C's safety belt: a candidate block becomes active when one of
// its (up to 26) neighbours was active in the previous round; neighbours wrap across
// periodic faces and do not exist beyond other faces. The first pass only inverts
// the candidate flags.
__global__ void activate_kernel(ActParams p) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < p.nblocks; b += gridDim.x * blockDim.x) {
    if (p.first) { p.out[b] = p.in[b] ? 0 : 1; continue; }
    unsigned char a = p.in[b];
    if (!a) {
      const DomDev& dm = p.doms[p.bdom[b]];
      const int l = b - dm.block0;
      const int i[3] = {l % dm.nb[0], (l / dm.nb[0]) % dm.nb[1], l / (dm.nb[0] * dm.nb[1])};
      int lo[3], hi[3];
#pragma unroll
      for (int k = 0; k < 3; k++) { lo[k] = dm.nb[k] > 1 ? -1 : 0; hi[k] = -lo[k]; }
      for (int oz = lo[2]; oz <= hi[2] && !a; oz++)
        for (int oy = lo[1]; oy <= hi[1] && !a; oy++)
          for (int ox = lo[0]; ox <= hi[0] && !a; ox++) {
            const int o[3] = {ox, oy, oz};
            int j[3];
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 3; k++) {
              j[k] = i[k] + o[k];
              if (j[k] < 0 || j[k] >= dm.nb[k]) {
                if (dm.bc[k][0] == 0) j[k] = j[k] < 0 ? j[k] + dm.nb[k] : j[k] - dm.nb[k];
                else ok = false;
              }
            }
            if (ok && p.in[dm.block0 + (j[2] * dm.nb[1] + j[1]) * dm.nb[0] + j[0]]) a = 1;
          }
    }
    p.out[b] = a;
  }
}

// Steady-state criterion over cell items; flag[] was set to 1 beforehand. NaN counts as
// a deviation.
__global__ void __launch_bounds__(256) flag_steady_kernel(FlagParams p) {
  for (int it = blockIdx.x; it < p.nitems; it += gridDim.x) {
    const CellItem ci = p.items[it];
    AMRFD_GUARD(p.err, cell_item_ok(p.doms, p.ndom, ci), continue)
    const DomDev dm = load_dom(p.doms + ci.dom);
    int o[3];
    block_coords(dm, ci.blk, o);
    int dev = 0;
    for (int c = threadIdx.x; c < ci.cnt && !dev; c += blockDim.x) {
      const int l = ci.c0 + c;
      const int lx = l % dm.be[0], ly = (l / dm.be[0]) % dm.be[1], lz = l / (dm.be[0] * dm.be[1]);
      const long long idx = dm.off + ((long long)(o[2] + lz) * dm.n[1] + (o[1] + ly)) * dm.n[0] + (o[0] + lx);
      for (int v = 0; v < p.nv; v++) {
        const long long e = idx + (long long)v * dm.ncell;
        if (!(fabs(p.U[e] - p.R[e]) <= p.tol)) { dev = 1; break; }
      }
    }
    if (__syncthreads_or(dev) && threadIdx.x == 0) p.flag[dm.block0 + ci.blk] = 0;
  }
}

cudaError_t launch_activate(const ActParams& p, cudaStream_t s) {
  const int grid = p.nblocks > 0 ? (p.nblocks + 255) / 256 : 1;
  activate_kernel<<<grid < 1024 ? grid : 1024, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_flag_steady(const FlagParams& p, int grid, cudaStream_t s) {
  flag_steady_kernel<<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_dt(const DtParams& p, cudaStream_t s) {
  dt_kernel<<<1, 1024, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_compact(const CompactParams& p, cudaStream_t s) {
  compact_scan_kernel<<<1, 1024, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n = p.list.ngroups;
  compact_copy_kernel<<<n < 4096 ? (n > 0 ? n : 1) : 4096, 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace amrfd
