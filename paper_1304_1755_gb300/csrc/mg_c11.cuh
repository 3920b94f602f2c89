// Constant-coefficient V(1,1) level kernels (abar = 1: every level carries the Q1
// stencil), included by k_mg.cu after mg_kernels.cuh.
//
// With c = omega / (8/3) and A = 3 I - S9/3 (S9 = 3 x 3 box sum) the fused level
// operations are separable filters:
//   down:  b_c = P^T (b - A c b) = (1 - 3c) (r3 (x) r3) b + (c/3) (r5 (x) r5) b,
//          r3 = (1/2, 1, 1/2), r5 = r3 * (1,1,1) = (1/2, 3/2, 2, 3/2, 1/2), centred on the
//          fine node 2I+1 that carries coarse node I;
//   up:    x = c b + e (e = P x_c) followed by one Jacobi step:
//          x' = (2c - 3c^2) b + (1 - 3c) e + S9 g,   g = (c^2/3) b + (c/3) e.
// A warp owns 32 coarse columns (down) or 64 fine columns (up) and walks down a strip of
// rows: horizontal neighbours come from warp shuffles, vertical ones from a sliding
// window in registers, and the loads of the next rows are issued two steps ahead so
// enough bytes are in flight to stream from HBM.  No shared memory, no barriers.
#pragma once

namespace {
constexpr int SLIDE_ROWS = 16;       // max coarse rows per warp strip (down); the up strip has 2x fine rows
constexpr int SLIDE_WARPS = 8;

template <typename TB, typename TA>
__device__ __forceinline__ TA ldz(const TB* p, bool ok) { return ok ? ld_as<TA>(p) : TA(0); }

template <typename TA> struct DRaw { TA v1, v2, l1, l2, r1; };

template <typename TB, typename TS, typename TA>
__global__ void __launch_bounds__(32 * SLIDE_WARPS) mg_down_slide(const TB* __restrict__ b, TS* __restrict__ bc,
                                                                  int m, int mc, size_t ldb, size_t ldc, TA c,
                                                                  int strips_x, int nstrips, int srows) {
  const int lane = threadIdx.x & 31;
  const int strip = blockIdx.x * SLIDE_WARPS + (threadIdx.x >> 5);
  if (strip >= nstrips) return;                    // uniform per warp
  const int sx = strip % strips_x, sy = strip / strips_x;
  const int I = sx * 32 + lane, J0 = sy * srows, J1 = min(J0 + srows, mc);
  const TB* bb = b + (size_t)blockIdx.y * ldb;
  TS* cb = bc + (size_t)blockIdx.y * ldc;
  // this lane's fine columns 2I+1, 2I+2; lane 0 also 2I-1, 2I; lane 31 also 2I+3
  const int c1 = 2 * I + 1;
  const bool ok1 = c1 < m, ok2 = c1 + 1 < m;
  const bool okl1 = lane == 0 && c1 - 2 >= 0 && c1 - 2 < m, okl2 = lane == 0 && c1 - 1 >= 0 && c1 - 1 < m;
  const bool okr = lane == 31 && c1 + 2 < m;
  const TA a3 = TA(1) - TA(3) * c, a5 = c / TA(3);
  auto load = [&](int r) {
    DRaw<TA> q;
    const bool rok = r >= 0 && r < m;
    const TB* rp = bb + (size_t)(rok ? r : 0) * m;
    q.v1 = ldz<TB, TA>(rp + c1, rok && ok1);
    q.v2 = ldz<TB, TA>(rp + c1 + 1, rok && ok2);
    q.l1 = ldz<TB, TA>(rp + c1 - 2, rok && okl1);
    q.l2 = ldz<TB, TA>(rp + c1 - 1, rok && okl2);
    q.r1 = ldz<TB, TA>(rp + c1 + 2, rok && okr);
    return q;
  };
  auto filt = [&](const DRaw<TA>& q, TA& s3, TA& s5) {
    TA l1 = __shfl_up_sync(0xffffffffu, q.v1, 1), l2 = __shfl_up_sync(0xffffffffu, q.v2, 1);
    TA r1 = __shfl_down_sync(0xffffffffu, q.v1, 1);
    if (lane == 0) l1 = q.l1, l2 = q.l2;
    if (lane == 31) r1 = q.r1;
    s3 = TA(0.5) * (l2 + q.v2) + q.v1;
    s5 = TA(0.5) * (l1 + r1) + TA(1.5) * (l2 + q.v2) + TA(2) * q.v1;
  };
  // rows 2J-1 .. 2J+3 around fine row 2J+1 of coarse row J
  TA h3[5], h5[5];
  {
    DRaw<TA> q[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) q[k] = load(2 * J0 - 1 + k);
#pragma unroll
    for (int k = 0; k < 5; ++k) filt(q[k], h3[k], h5[k]);
  }
  DRaw<TA> pa = load(2 * J0 + 4), pb = load(2 * J0 + 5), pc = load(2 * J0 + 6), pd = load(2 * J0 + 7);
  for (int J = J0; J < J1; ++J) {
    if (I < mc) {
      const TA v3 = TA(0.5) * (h3[1] + h3[3]) + h3[2];
      const TA v5 = TA(0.5) * (h5[0] + h5[4]) + TA(1.5) * (h5[1] + h5[3]) + TA(2) * h5[2];
      st_as<TS, TA>(cb + (size_t)J * mc + I, a3 * v3 + a5 * v5);
    }
    if (J + 1 < J1) {
      h3[0] = h3[2], h3[1] = h3[3], h3[2] = h3[4];
      h5[0] = h5[2], h5[1] = h5[3], h5[2] = h5[4];
      filt(pa, h3[3], h5[3]);
      filt(pb, h3[4], h5[4]);
      pa = pc, pb = pd;
      if (J + 2 < J1) pc = load(2 * J + 8), pd = load(2 * J + 9);
    }
  }
}

// up: lane fine columns i0 = X0 + 2 lane (even interior index: between coarse C-1 and C) and
// i1 = i0 + 1 (odd: on coarse C), C = X0/2 + lane; halo columns X0 - 1 (lane 0, on C - 1) and
// X0 + 64 (lane 31, between C and C + 1).  Fine row j lies between coarse rows (j-1)>>1 and j>>1.
template <typename TA> struct URawB { TA b0, b1, bh; };
template <typename TA> struct URawC { TA own, left, right; };

template <typename TB, typename TS, typename TA>
__global__ void __launch_bounds__(32 * SLIDE_WARPS) mg_up_slide(const TB* __restrict__ b, const TS* __restrict__ xc,
                                                                TS* __restrict__ x, int m, int mc, size_t ldb,
                                                                size_t ldc, size_t ldx, TA c, int strips_x,
                                                                int nstrips, int srows) {
  const int lane = threadIdx.x & 31;
  const int strip = blockIdx.x * SLIDE_WARPS + (threadIdx.x >> 5);
  if (strip >= nstrips) return;
  const int sx = strip % strips_x, sy = strip / strips_x;
  const int X0 = sx * 64, Y0 = sy * (2 * srows), Y1 = min(Y0 + 2 * srows, m);
  const TB* bb = b + (size_t)blockIdx.y * ldb;
  const TS* xcb = xc + (size_t)blockIdx.y * ldc;
  TS* xb = x + (size_t)blockIdx.y * ldx;
  const int i0 = X0 + 2 * lane, i1 = i0 + 1, C = (X0 >> 1) + lane;
  const bool ok0 = i0 < m, ok1 = i1 < m;
  const bool okC = C < mc, okCm = lane == 0 && C - 1 >= 0 && C - 1 < mc;
  const bool okhl = lane == 0 && X0 - 1 >= 0, okhr = lane == 31 && X0 + 64 < m;
  const bool okCr = lane == 31 && C + 1 < mc;
  const int hcol = lane == 0 ? X0 - 1 : X0 + 64;
  const bool okh = okhl || okhr;
  const TA cgb = c * c / TA(3), cge = c / TA(3), cbb = TA(2) * c - TA(3) * c * c, cee = TA(1) - TA(3) * c;
  auto load_b = [&](int j) {
    URawB<TA> q;
    const bool jok = j >= 0 && j < m;
    const TB* rp = bb + (size_t)(jok ? j : 0) * m;
    q.b0 = ldz<TB, TA>(rp + i0, jok && ok0);
    q.b1 = ldz<TB, TA>(rp + i1, jok && ok1);
    q.bh = ldz<TB, TA>(rp + hcol, jok && okh);
    return q;
  };
  auto load_c = [&](int R) {
    URawC<TA> q;
    const bool rok = R >= 0 && R < mc;
    const TS* rp = xcb + (size_t)(rok ? R : 0) * mc;
    q.own = ldz<TS, TA>(rp + C, rok && okC);
    q.left = ldz<TS, TA>(rp + C - 1, rok && okCm);
    q.right = ldz<TS, TA>(rp + C + 1, rok && okCr);
    return q;
  };
  // horizontal 3-sums of g and the (cb b + ce e) terms of fine row j from its raw data and the
  // coarse rows below / above it (equal for odd j)
  auto frow = [&](int j, const URawB<TA>& qb, const URawC<TA>& ca, const URawC<TA>& cbr, TA& H0, TA& H1,
                  TA& be0, TA& be1) {
    const bool jok = j >= 0 && j < m;
    const TA wa = (j & 1) ? TA(1) : TA(0.5), wb = (j & 1) ? TA(0) : TA(0.5);
    const TA own = wa * ca.own + wb * cbr.own;
    TA left = __shfl_up_sync(0xffffffffu, own, 1);
    if (lane == 0) left = wa * ca.left + wb * cbr.left;
    const TA right = wa * ca.right + wb * cbr.right;          // used by lane 31 only
    const TA e1 = own, e0 = TA(0.5) * (left + own);
    const TA g0 = jok && ok0 ? cgb * qb.b0 + cge * e0 : TA(0);
    const TA g1 = jok && ok1 ? cgb * qb.b1 + cge * e1 : TA(0);
    TA gl = __shfl_up_sync(0xffffffffu, g1, 1), gr = __shfl_down_sync(0xffffffffu, g0, 1);
    if (lane == 0) gl = jok && okhl ? cgb * qb.bh + cge * left : TA(0);
    if (lane == 31) gr = jok && okhr ? cgb * qb.bh + cge * TA(0.5) * (own + right) : TA(0);
    H0 = (gl + g0) + g1;
    H1 = (g0 + g1) + gr;
    be0 = cbb * qb.b0 + cee * e0;
    be1 = cbb * qb.b1 + cee * e1;
  };
  // coarse rows needed by fine row j: (j-1)>>1 and j>>1; keep the window (Rb, Rb+1, Rb+2) with Rb
  // the lower coarse row of the current fine row
  int Rb = (Y0 - 2) >> 1;                                       // lower coarse row of fine row Y0 - 1
  URawC<TA> c0 = load_c(Rb), c1 = load_c(Rb + 1), c2 = load_c(Rb + 2), c3 = load_c(Rb + 3);
  URawB<TA> bm = load_b(Y0 - 1), bcur = load_b(Y0), bn1 = load_b(Y0 + 1), bn2 = load_b(Y0 + 2);
  auto coarse_pair = [&](int j, URawC<TA>& a, URawC<TA>& bq) {
    const int lo = (j - 1) >> 1, hi = j >> 1;
    a = (lo == Rb) ? c0 : ((lo == Rb + 1) ? c1 : c2);
    bq = (hi == Rb) ? c0 : ((hi == Rb + 1) ? c1 : ((hi == Rb + 2) ? c2 : c3));
  };
  TA Hm0, Hm1, Hc0, Hc1, Hp0, Hp1, be0, be1, bn0v, bn1v, t0, t1;
  {
    URawC<TA> a, bq;
    coarse_pair(Y0 - 1, a, bq);
    frow(Y0 - 1, bm, a, bq, Hm0, Hm1, t0, t1);
    coarse_pair(Y0, a, bq);
    frow(Y0, bcur, a, bq, Hc0, Hc1, be0, be1);
  }
  for (int j = Y0; j < Y1; ++j) {
    // shift the coarse window so that it starts at the lower coarse row of fine row j + 1
    if (((j) >> 1) > Rb + 1 || ((j + 1 - 1) >> 1) > Rb) {
      c0 = c1, c1 = c2, c2 = c3;
      ++Rb;
      c3 = load_c(Rb + 3);
    }
    URawC<TA> a, bq;
    coarse_pair(j + 1, a, bq);
    frow(j + 1, bn1, a, bq, Hp0, Hp1, bn0v, bn1v);
    bn1 = bn2;
    bn2 = load_b(j + 3);
    TS* op = xb + (size_t)j * m;
    if (ok0) st_as<TS, TA>(op + i0, be0 + ((Hm0 + Hc0) + Hp0));
    if (ok1) st_as<TS, TA>(op + i1, be1 + ((Hm1 + Hc1) + Hp1));
    Hm0 = Hc0, Hm1 = Hc1, Hc0 = Hp0, Hc1 = Hp1, be0 = bn0v, be1 = bn1v;
  }
}
}  // namespace
