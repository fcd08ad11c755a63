// amrfd_adjoint.cu -- discrete adjoint of one SSPRK step of the FD-MP5 update.
//
// With the splitting speeds c_max (per stage), the GLM speed c_h and the psi
// damping factor held at their forward values, one stage is
//   U^(i) = sum_t a_t U^(k_t) + sum_d w_d D_d(S),   S = U^(i-1), w_d = dt b / (2 dx_d),
// where D_d(S)_j = Fsum_j - Fsum_{j+1} and Fsum_k = G+_{k-1} + G-_k + (Y+_k + Y-_k)/2
// is the interface flux of Sec. 2.2 in units of 2 F^ (G = F +- c_max U). Every MP5
// value Y is piecewise linear in its stencil once the limiter's choices are fixed;
// the forward recomputation records, per face, variable and bias, which pieces the
// limiter took (a 9-bit tape), and the adjoint applies their transposes without
// re-evaluating the limiter. Gradients are gathered per cell (no atomics):
// a segment recomputes the faces within reach of its cells (two beyond on the low
// side, three on the high side) and keeps only contributions to its own cells;
// with outflow faces the ghost copies of an edge cell fold back into it.
#include <cuda_runtime.h>

#include "amrfd_device.cuh"
#include "amrfd_kernels.cuh"

namespace amrfd {

// Transposed flux-split Jacobian: gu = (dG+/dU)^T gp + (dG-/dU)^T gm with
// G+- = F_D(U) +- alpha U (alpha, c_h fixed).
template <int PHYS, int NV, int D>
__device__ __forceinline__ void split_flux_adj(const double* u, double gm1, double alpha, double ch2,
                                               const double* gp, const double* gmn, double* gu) {
  double y[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) {
    y[v] = gp[v] + gmn[v];
    gu[v] = alpha * (gp[v] - gmn[v]);
  }
  const double rho = u[0];
  const double ir = frcp(rho);
  if (PHYS == PH_EULER) {
    constexpr int nm = NV - 2;
    double v[nm], gv[nm];
    double mv = 0.0;
#pragma unroll
    for (int k = 0; k < nm; k++) { v[k] = u[1 + k] * ir; mv = fma(u[1 + k], v[k], mv); gv[k] = 0.0; }
    const double E = u[NV - 1];
    const double p = gm1 * fma(-0.5, mv, E);
    const double vd = v[D];
    double gp_ = 0.0, gE = 0.0;
    gu[1 + D] += y[0];
#pragma unroll
    for (int k = 0; k < nm; k++) {
      gv[D] += y[1 + k] * u[1 + k];
      gu[1 + k] += y[1 + k] * vd;
      if (k == D) gp_ += y[1 + k];
    }
    gv[D] += y[NV - 1] * (E + p);
    gE += y[NV - 1] * vd;
    gp_ += y[NV - 1] * vd;
    gE += gm1 * gp_;
    const double gmv = -0.5 * gm1 * gp_;
    double gir = 0.0;
#pragma unroll
    for (int k = 0; k < nm; k++) {
      gu[1 + k] += gmv * v[k];
      gv[k] += gmv * u[1 + k];
      gu[1 + k] += gv[k] * ir;
      gir += gv[k] * u[1 + k];
    }
    gu[0] -= gir * ir * ir;
    gu[NV - 1] += gE;
  } else {
    const double E = u[4];
    const double B[3] = {u[5], u[6], u[7]};
    const double v[3] = {u[1] * ir, u[2] * ir, u[3] * ir};
    const double b2 = fma(B[2], B[2], fma(B[1], B[1], B[0] * B[0]));
    const double mv = fma(u[3], v[2], fma(u[2], v[1], u[1] * v[0]));
    const double p = gm1 * fma(-0.5, mv + b2, E);
    const double ptot = fma(0.5, b2, p);
    const double vb = fma(v[2], B[2], fma(v[1], B[1], v[0] * B[0]));
    const double vd = v[D], bd = B[D];
    double gv[3] = {0.0, 0.0, 0.0}, gB[3] = {0.0, 0.0, 0.0};
    double gptot = 0.0, gE = 0.0, gvb = 0.0, gpsi = 0.0;
    gu[1 + D] += y[0];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const double yk = y[1 + k];
      gv[D] += yk * u[1 + k];
      gu[1 + k] += yk * vd;
      gB[D] -= yk * B[k];
      gB[k] -= yk * bd;
      if (k == D) gptot += yk;
    }
    gv[D] += y[4] * (E + ptot);
    gE += y[4] * vd;
    gptot += y[4] * vd;
    gB[D] -= y[4] * vb;
    gvb -= y[4] * bd;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const double yk = y[5 + k];
      if (k == D) {
        gpsi += yk;
      } else {
        gv[D] += yk * B[k];
        gB[k] += yk * vd;
        gB[D] -= yk * v[k];
        gv[k] -= yk * bd;
      }
    }
    gB[D] += y[8] * ch2;
#pragma unroll
    for (int k = 0; k < 3; k++) { gv[k] += gvb * B[k]; gB[k] += gvb * v[k]; }
    double gb2 = 0.5 * gptot;
    const double gp_ = gptot;
    gE += gm1 * gp_;
    const double gmv = -0.5 * gm1 * gp_;
    gb2 -= 0.5 * gm1 * gp_;
    double gir = 0.0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      gu[1 + k] += gmv * v[k];
      gv[k] += gmv * u[1 + k];
      gB[k] += 2.0 * B[k] * gb2;
      gu[1 + k] += gv[k] * ir;
      gir += gv[k] * u[1 + k];
      gu[5 + k] += gB[k];
    }
    gu[0] -= gir * ir * ir;
    gu[4] += gE;
    gu[8] += gpsi;
  }
}

// Backward of one reconstruction at face k for one variable, from the recorded
// pieces: rec = (piece of the MP5 value) | (piece of Mp) << 3 | (piece of Mm) << 6.
// The stencil occupies positions q0..q0+4 of the line window; NEG is the mirrored
// (right-biased) reconstruction. Accumulates d(value)/dG * gY into gG.
// The weights of the unlimited value as register operands: 4, 6, 26, 54 (/60).
struct FaceW {
  double a4, a6, a26, a54;
};

template <bool NEG>
__device__ __forceinline__ void face_adj(double* gG, int q0, double gY, unsigned rec, const FaceW& fw) {
  if ((rec & 7) == SEL_X) {
    // the unlimited value f_or (the common case): fixed weights on the five G values,
    // the differences' coefficients (-4, 22, 48, -6)/60 telescoped (mirrored for NEG)
    gG[q0] = fma(NEG ? -fw.a6 : fw.a4, gY, gG[q0]);
    gG[q0 + 1] = fma(NEG ? fw.a54 : -fw.a26, gY, gG[q0 + 1]);
    gG[q0 + 2] = fma(-fw.a26, gY, gG[q0 + 2]);
    gG[q0 + 3] = fma(NEG ? -fw.a26 : fw.a54, gY, gG[q0 + 3]);
    gG[q0 + 4] = fma(NEG ? fw.a4 : -fw.a6, gY, gG[q0 + 4]);
    return;
  }
  double gDm, gD0, gD1, gDp, gMp, gMm;
  if (!NEG) mp5_rel2_grad<false>(rec & 7, gY, gDm, gD0, gD1, gDp, gMp, gMm);
  else mp5_rel2_grad<true>(rec & 7, gY, gDm, gD0, gD1, gDp, gMp, gMm);
  // curvatures kL, kC, kR at q0+1, q0+2, q0+3 (line order)
  double gkL = 0.0, gkC = 0.0, gkR = 0.0, t1, t2;
  if (!NEG) {
    dm4_grad((rec >> 6) & 7, gMm, t1, t2); gkL += t1; gkC += t2;  // Mm from (kL, kC)
    dm4_grad((rec >> 3) & 7, gMp, t1, t2); gkC += t1; gkR += t2;  // Mp from (kC, kR)
  } else {
    dm4_grad((rec >> 3) & 7, gMp, t1, t2); gkL += t1; gkC += t2;  // mirrored: Mp from (kL, kC)
    dm4_grad((rec >> 6) & 7, gMm, t1, t2); gkC += t1; gkR += t2;  // Mm from (kC, kR)
  }
  // gradients of the line differences h_j = G[q0+j] - G[q0+j-1], j = 1..4
  double gh1, gh2, gh3, gh4;
  if (!NEG) { gh1 = gDm; gh2 = gD0; gh3 = gD1; gh4 = gDp; }
  else { gh1 = gDp; gh2 = gD1; gh3 = gD0; gh4 = gDm; }
  // kL = h2 - h1, kC = h3 - h2, kR = h4 - h3
  gh1 -= gkL; gh2 += gkL - gkC; gh3 += gkC - gkR; gh4 += gkR;
  gG[q0] -= gh1;
  gG[q0 + 1] += gh1 - gh2;
  gG[q0 + 2] += gh2 - gh3;
  gG[q0 + 3] += gh3 - gh4;
  gG[q0 + 4] += gh4;
}

// Whether the block next to block `blk` along d (side -1 or +1) exists and is active
// (wrapping across periodic faces).
__device__ __forceinline__ bool nb_active(const DomDev& dm, const unsigned char* active, int blk, int d, int side) {
  const int bi[3] = {blk % dm.nb[0], (blk / dm.nb[0]) % dm.nb[1], blk / (dm.nb[0] * dm.nb[1])};
  int j = bi[d] + side;
  if (j < 0 || j >= dm.nb[d]) {
    if (dm.bc[d][0] != 0) return false;
    j = j < 0 ? j + dm.nb[d] : j - dm.nb[d];
  }
  const int stride = d == 0 ? 1 : (d == 1 ? dm.nb[0] : dm.nb[0] * dm.nb[1]);
  return active[dm.block0 + blk + (j - bi[d]) * stride] != 0;
}

// A passive block whose cells fed an active neighbour's fluxes along d: the active cells'
// faces reach three cells into it (blocks hold at least three cells along d when their
// domain is partly active), where the forward pass read U^n.
__device__ __forceinline__ bool passive_fed(const DomDev& dm, const unsigned char* active, int blk, int d) {
  return !active[dm.block0 + blk] && (nb_active(dm, active, blk, d, -1) || nb_active(dm, active, blk, d, 1));
}

// Backward of one LIMO3 value Y(a, b) at a face from its recorded piece (limo3_y_sel):
// dY/da, dY/db of the piece. Inside the 2e-12-wide blend band of the switch the exact
// derivative carries a factor 1e12 through the blend weight; there the piece of the
// nearer half (unlimited or limited) is taken.
__device__ __forceinline__ void limo3_piece_grad(unsigned rec, double& ca, double& cb) {
  const unsigned mode = (rec >> 3) & 3u;
  if (mode == 0u || mode == 2u) { ca = 1.0 / 3.0; cb = 2.0 / 3.0; return; }
  switch (rec & 7u) {
    case 1: ca = 1.0 / 3.0; cb = 2.0 / 3.0; break;  // y3
    case 2: ca = -0.5; cb = 0.0; break;               // -a/2
    case 3: ca = 2.0; cb = 0.0; break;                // 2a
    case 4: ca = 0.0; cb = 1.6; break;                // 1.6 b
    default: ca = 0.0; cb = 0.0; break;               // zero
  }
}

template <int PHYS, int NV, int D>
__device__ __forceinline__ void adj_item(const AdjFluxParams& p, const FluxItem& it, double* sm) {
  constexpr int od1 = D == 0 ? 1 : 0;
  constexpr int od2 = D == 2 ? 1 : 2;
  const DomDev dm = *(p.doms + it.dom);
  int o[3];
  {
    const int bx = it.blk % dm.nb[0], by = (it.blk / dm.nb[0]) % dm.nb[1], bz = it.blk / (dm.nb[0] * dm.nb[1]);
    o[0] = bx * dm.be[0]; o[1] = by * dm.be[1]; o[2] = bz * dm.be[2];
  }
  const unsigned long long* sk = p.araw + (size_t)it.dom * 4;
  const unsigned long long* s0p = p.araw0 + (size_t)it.dom * 4;
  double ch = 0.0;
  if (p.glm)
    for (int d = 0; d < p.ndim; d++) ch = imax(ch, bitsd((long long)s0p[d]));
  const double alpha = imax(bitsd((long long)sk[D]), ch);
  const double ch2 = ch * ch;
  const double w = p.dt[it.dom] * p.b * (0.5 / dm.dx[D]);
  const double pfac = p.psi_fac ? p.psi_fac[it.dom] : 1.0;
  const int nl = it.nl, slen = it.slen, P = p.P, SA = p.SSa, SG = p.SSg;
  const int n = dm.n[D];
  const int s0 = o[D] + it.s0;               // first cell of the segment (domain coordinate)
  const int WA = slen + 10, WG = slen + 6;
  double* gGp = sm;                           // [NV][P][SA] gradient w.r.t. G+ at positions s0-5 ..
  double* gGm = gGp + NV * P * SA;
  double* gh = gGm + NV * P * SA;             // [NV][P][SG] scaled upstream gradient at s0-3 ..
  // passive block (fed an active neighbour): its cells entered the fluxes as U^n
  const bool self_active = p.active[dm.block0 + it.blk] != 0;
  const int bstride = D == 0 ? 1 : (D == 1 ? dm.nb[0] : dm.nb[0] * dm.nb[1]);
  const int bo = it.blk - (o[D] / dm.be[D]) * bstride;  // block index with coordinate D = 0
  // ---- phase A: upstream gradient at s0-3 .. s0+slen+2 (zero beyond an outflow face and
  // at passive cells, whose residual the step does not use)
  for (int c = threadIdx.x; c < nl * WA; c += blockDim.x) {
    int pl, q;
    if (D == 0) { pl = c / WA; q = c - pl * WA; }
    else { q = c / nl; pl = c - q * nl; }
#pragma unroll
    for (int v = 0; v < NV; v++) {
      gGp[(v * P + pl) * SA + q] = 0.0;
      gGm[(v * P + pl) * SA + q] = 0.0;
    }
    const int r = q - 2;
    if (r < 0 || r >= WG) continue;
    const int line = it.l0 + pl;
    const int a1 = line % dm.be[od1], a2 = line / dm.be[od1];
    int x[3];
    x[od1] = o[od1] + a1;
    x[od2] = o[od2] + a2;
    int g = s0 - 3 + r;
    bool live = true;
    if (g < 0) { live = dm.bc[D][0] == 0; g = ((g % n) + n) % n; }
    else if (g >= n) { live = dm.bc[D][1] == 0; g = g % n; }
    x[D] = g;
    live = live && p.active[dm.block0 + bo + (g / dm.be[D]) * bstride] != 0;
    const long long idx = ((long long)x[2] * dm.n[1] + x[1]) * dm.n[0] + x[0];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      double gv = 0.0;
      if (live) {
        gv = p.G[dm.off + idx + (long long)v * dm.ncell] * w;
        if (PHYS == PH_MHD && v == 8) gv *= pfac;
      }
      gh[(v * P + pl) * SG + r] = gv;
    }
  }
  __syncthreads();
  // ---- phase B: one thread per (line, variable) walks the faces within reach
  int kb = s0 - 2, ke = s0 + slen + 2;
  if (dm.bc[D][0] != 0 && kb < 0) kb = 0;
  if (dm.bc[D][1] != 0 && ke > n) ke = n;
  const long long nlines = (long long)dm.n[od1] * dm.n[od2];
  const double one = ldk(K_ONE), half = ldk(K_HALF), mz = ldk(K_MZ);
  const FaceW fw = {ldk(K_C4), ldk(K_C6), ldk(K_C26), ldk(K_C54)};
  for (int t = threadIdx.x; t < nl * NV; t += blockDim.x) {
    const int v = t / nl, pl = t - v * nl;
    double* ggp = gGp + (v * P + pl) * SA;
    double* ggm = gGm + (v * P + pl) * SA;
    const double* ghl = gh + (v * P + pl) * SG;
    const int line = it.l0 + pl;
    const int a1 = line % dm.be[od1], a2 = line / dm.be[od1];
    const long long ld = (long long)(o[od2] + a2) * dm.n[od1] + (o[od1] + a1);
    const unsigned short* tp = p.tape + dm.tape_off[D] + ((long long)(v * 2 + 0) * nlines + ld) * (n + 1);
    const unsigned short* tm = p.tape + dm.tape_off[D] + ((long long)(v * 2 + 1) * nlines + ld) * (n + 1);
    for (int k = kb; k <= ke; k++) {
      const int qk = k - (s0 - 5);        // position of cell k in the G window
      const int rk = k - (s0 - 3);        // position of cell k in the gradient window
      const double gF = rsub(ghl[rk], ghl[rk - 1], one);
      if (abits(gF) == 0) continue;
      const int f = (k < 0) ? k + n : (k >= n && dm.bc[D][1] == 0 ? k - n : k);  // periodic faces wrap
      ggp[qk - 1] = radd(ggp[qk - 1], gF, one);
      ggm[qk] = radd(ggm[qk], gF, one);
      const double gY = rmul(half, gF, mz);
      if (p.limo3) {
        // F = G+_{k-1} + G-_k + (Y+ - Y-)/2: Y+ of a = G+_{k-1} - G+_{k-2}, b = G+_k - G+_{k-1};
        // Y- of a = G-_{k+1} - G-_k, b = G-_k - G-_{k-1}
        double ca, cb;
        limo3_piece_grad(tp[f], ca, cb);
        ggp[qk - 2] -= ca * gY;
        ggp[qk - 1] += (ca - cb) * gY;
        ggp[qk] += cb * gY;
        limo3_piece_grad(tm[f], ca, cb);
        ggm[qk + 1] -= ca * gY;
        ggm[qk] += (ca - cb) * gY;
        ggm[qk - 1] += cb * gY;
      } else {
        face_adj<false>(ggp, qk - 3, gY, tp[f], fw);  // + stencil: cells k-3 .. k+1, centre k-1
        face_adj<true>(ggm, qk - 2, gY, tm[f], fw);   // - stencil: cells k-2 .. k+2, centre k
      }
    }
    // outflow: ghost copies of an edge cell fold back into it
    if (dm.bc[D][0] == 1 && s0 == 0) {
      const int q0 = 5;  // position of cell 0
      for (int qq = 2; qq < q0; qq++) { ggp[q0] += ggp[qq]; ggm[q0] += ggm[qq]; }
    }
    if (dm.bc[D][1] == 1 && s0 + slen == n) {
      const int qn = slen + 4;  // position of cell n-1
      for (int qq = qn + 1; qq <= qn + 3; qq++) { ggp[qn] += ggp[qq]; ggm[qn] += ggm[qq]; }
    }
  }
  __syncthreads();
  // ---- phase C: transposed flux-split Jacobian per cell of the segment
  for (int c = threadIdx.x; c < nl * slen; c += blockDim.x) {
    int pl, j;
    if (D == 0) { pl = c / slen; j = c - pl * slen; }
    else { j = c / nl; pl = c - j * nl; }
    const int line = it.l0 + pl;
    const int a1 = line % dm.be[od1], a2 = line / dm.be[od1];
    int x[3];
    x[od1] = o[od1] + a1;
    x[od2] = o[od2] + a2;
    x[D] = s0 + j;
    const long long idx = ((long long)x[2] * dm.n[1] + x[1]) * dm.n[0] + x[0];
    double u[NV], gpv[NV], gmv[NV], gu[NV];
    const double* Sv = self_active ? p.S : p.Un;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      u[v] = Sv[dm.off + idx + (long long)v * dm.ncell];
      gpv[v] = gGp[(v * P + pl) * SA + j + 5];
      gmv[v] = gGm[(v * P + pl) * SA + j + 5];
    }
    split_flux_adj<PHYS, NV, D>(u, p.gm1, alpha, ch2, gpv, gmv, gu);
    // mirror faces: the ghost image of this cell (odd variables negated) fed the
    // split fluxes too; its gradient goes through the Jacobian at the image state
    // and back through the sign flip (the segment at a mirror face holds >= 3 cells)
    for (int side = 0; side < 2; side++) {
      int q = -1;
      if (side == 0 && dm.bc[D][0] == 2 && s0 == 0 && j < 3) q = 4 - j;
      if (side == 1 && dm.bc[D][1] == 2 && s0 + slen == n && j >= slen - 3) q = 2 * slen + 4 - j;
      if (q < 0) continue;
      const unsigned odd = dm.asym[D][side];
      double ui[NV], gi[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) {
        ui[v] = ((odd >> v) & 1u) ? -u[v] : u[v];
        gpv[v] = gGp[(v * P + pl) * SA + q];
        gmv[v] = gGm[(v * P + pl) * SA + q];
      }
      split_flux_adj<PHYS, NV, D>(ui, p.gm1, alpha, ch2, gpv, gmv, gi);
#pragma unroll
      for (int v = 0; v < NV; v++) gu[v] += ((odd >> v) & 1u) ? -gi[v] : gi[v];
    }
#pragma unroll
    for (int v = 0; v < NV; v++) p.gL[D][dm.off + idx + (long long)v * dm.ncell] = gu[v];
  }
  __syncthreads();
}

template <int PHYS, int NV>
__global__ void __launch_bounds__(256) adj_flux_kernel(AdjFluxParams p) {
  extern __shared__ double sm[];
  constexpr int maxd = PHYS == PH_EULER ? NV - 2 : 3;
  for (int it = blockIdx.x; it < p.nitems; it += gridDim.x) {
    const FluxItem item = p.items[p.item0 + it];
    AMRFD_GUARD(p.err, flux_item_ok(p.doms, p.ndom, p.ndim, p.P, p.SSg, item), continue)
    {
      const DomDev& dm = p.doms[item.dom];
      if (!p.active[dm.block0 + item.blk] && !passive_fed(dm, p.active, item.blk, item.d)) continue;
    }
    if (item.d == 0) adj_item<PHYS, NV, 0>(p, item, sm);
    if constexpr (maxd > 1) { if (item.d == 1) adj_item<PHYS, NV, 1>(p, item, sm); }
    if constexpr (maxd > 2) { if (item.d == 2) adj_item<PHYS, NV, 2>(p, item, sm); }
  }
}

// Transposed stage combination: g[U^(k_t)] += a_t gOut, g[U^(i-1)] += sum_d gL_d.
template <int NV>
__global__ void __launch_bounds__(256) adj_combine_kernel(AdjCombParams p) {
  for (int it = blockIdx.x; it < p.nitems; it += gridDim.x) {
    const CellItem ci = p.items[p.item0 + it];
    AMRFD_GUARD(p.err, cell_item_ok(p.doms, p.ndom, ci), continue)
    const DomDev dm = p.doms[ci.dom];
    int o[3];
    {
      const int bx = ci.blk % dm.nb[0], by = (ci.blk / dm.nb[0]) % dm.nb[1], bz = ci.blk / (dm.nb[0] * dm.nb[1]);
      o[0] = bx * dm.be[0]; o[1] = by * dm.be[1]; o[2] = bz * dm.be[2];
    }
    if (!p.active[dm.block0 + ci.blk]) {
      // a passive block's cells entered the stage's fluxes as U^n where they fed an
      // active neighbour: those directions' gradients belong to U^n
      bool fed[3];
      bool any = false;
      for (int d = 0; d < 3; d++) {
        fed[d] = d < p.ndim && passive_fed(dm, p.active, ci.blk, d);
        any |= fed[d];
      }
      if (!any) continue;
      for (int c = threadIdx.x; c < ci.cnt; c += blockDim.x) {
        const int l = ci.c0 + c;
        const int lx = l % dm.be[0], ly = (l / dm.be[0]) % dm.be[1], lz = l / (dm.be[0] * dm.be[1]);
        const long long idx = dm.off + ((long long)(o[2] + lz) * dm.n[1] + (o[1] + ly)) * dm.n[0] + (o[0] + lx);
#pragma unroll
        for (int v = 0; v < NV; v++) {
          const long long e = idx + (long long)v * dm.ncell;
          double s = 0.0;
          for (int d = 0; d < 3; d++)
            if (fed[d]) s += p.gL[d][e];
          p.gbuf[0][e] += s;
        }
      }
      continue;
    }
    const double pfac = p.psi_fac ? p.psi_fac[ci.dom] : 1.0;
    for (int c = threadIdx.x; c < ci.cnt; c += blockDim.x) {
      const int l = ci.c0 + c;
      const int lx = l % dm.be[0], ly = (l / dm.be[0]) % dm.be[1], lz = l / (dm.be[0] * dm.be[1]);
      const long long idx = dm.off + ((long long)(o[2] + lz) * dm.n[1] + (o[1] + ly)) * dm.n[0] + (o[0] + lx);
#pragma unroll
      for (int v = 0; v < NV; v++) {
        const long long e = idx + (long long)v * dm.ncell;
        double g = p.gout[e];
        if (NV == 9 && v == 8) g *= pfac;
        for (int t = 0; t < p.co.nterm; t++) p.gbuf[p.co.k[t]][e] = fma(p.co.a[t], g, p.gbuf[p.co.k[t]][e]);
        double s = p.gL[0][e];
        if (p.ndim > 1) s += p.gL[1][e];
        if (p.ndim > 2) s += p.gL[2][e];
        p.gbuf[p.kin][e] += s;
      }
    }
  }
}

// Passive blocks are the identity map of U^n: their gradient passes through (added to what
// the stages' fluxes gave U^n there, where the block fed an active neighbour).
__global__ void __launch_bounds__(256) adj_passive_kernel(AdjCombParams p) {
  for (int it = blockIdx.x; it < p.nitems; it += gridDim.x) {
    const CellItem ci = p.items[p.item0 + it];
    AMRFD_GUARD(p.err, cell_item_ok(p.doms, p.ndom, ci), continue)
    const DomDev dm = p.doms[ci.dom];
    if (p.active[dm.block0 + ci.blk]) continue;
    int o[3];
    {
      const int bx = ci.blk % dm.nb[0], by = (ci.blk / dm.nb[0]) % dm.nb[1], bz = ci.blk / (dm.nb[0] * dm.nb[1]);
      o[0] = bx * dm.be[0]; o[1] = by * dm.be[1]; o[2] = bz * dm.be[2];
    }
    for (int c = threadIdx.x; c < ci.cnt; c += blockDim.x) {
      const int l = ci.c0 + c;
      const int lx = l % dm.be[0], ly = (l / dm.be[0]) % dm.be[1], lz = l / (dm.be[0] * dm.be[1]);
      const long long idx = dm.off + ((long long)(o[2] + lz) * dm.n[1] + (o[1] + ly)) * dm.n[0] + (o[0] + lx);
      for (int v = 0; v < p.nv; v++) {
        const long long e = idx + (long long)v * dm.ncell;
        p.gbuf[0][e] += p.gout[e];
      }
    }
  }
}

// psi damping factor exp(-dt c_h / c_r) per domain, as applied by the forward step
__global__ void psi_fac_kernel(const unsigned long long* araw0, const double* dt, double* fac, int ndom, int ndim,
                               double cr, int glm) {
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < ndom; d += gridDim.x * blockDim.x) {
    double f = 1.0;
    if (glm && cr > 0.0) {
      double ch = 0.0;
      for (int k = 0; k < ndim; k++) ch = imax(ch, bitsd((long long)araw0[(size_t)d * 4 + k]));
      f = exp(-dt[d] * ch / cr);
    }
    fac[d] = f;
  }
}

#define AMRFD_DISPATCH_ADJ(physics, nv, CALL)                               \
  do {                                                                      \
    if ((physics) == PH_MHD && (nv) == 9) { CALL(PH_MHD, 9); }              \
    else if ((physics) == PH_EULER && (nv) == 3) { CALL(PH_EULER, 3); }     \
    else if ((physics) == PH_EULER && (nv) == 4) { CALL(PH_EULER, 4); }     \
    else if ((physics) == PH_EULER && (nv) == 5) { CALL(PH_EULER, 5); }     \
    else return cudaErrorInvalidValue;                                      \
  } while (0)

cudaError_t launch_adj_flux(int physics, int nv, const AdjFluxParams& p, int grid, int block, size_t smem,
                            cudaStream_t s) {
#define CALL(PH, NVV)                                                                                      \
  {                                                                                                        \
    cudaError_t e = cudaFuncSetAttribute(adj_flux_kernel<PH, NVV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                                                       \
    if (e != cudaSuccess) return e;                                                                        \
    adj_flux_kernel<PH, NVV><<<grid, block, smem, s>>>(p);                                                 \
  }
  AMRFD_DISPATCH_ADJ(physics, nv, CALL);
#undef CALL
  return cudaGetLastError();
}

cudaError_t launch_adj_combine(int nv, const AdjCombParams& p, int grid, int block, cudaStream_t s) {
  if (nv == 9) adj_combine_kernel<9><<<grid, block, 0, s>>>(p);
  else if (nv == 3) adj_combine_kernel<3><<<grid, block, 0, s>>>(p);
  else if (nv == 4) adj_combine_kernel<4><<<grid, block, 0, s>>>(p);
  else if (nv == 5) adj_combine_kernel<5><<<grid, block, 0, s>>>(p);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_adj_passive(const AdjCombParams& p, int grid, int block, cudaStream_t s) {
  adj_passive_kernel<<<grid, block, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_psi_fac(const unsigned long long* araw0, const double* dt, double* fac, int ndom, int ndim,
                           double cr, int glm, cudaStream_t s) {
  psi_fac_kernel<<<(ndom + 255) / 256, 256, 0, s>>>(araw0, dt, fac, ndom, ndim, cr, glm);
  return cudaGetLastError();
}

}  // namespace amrfd
