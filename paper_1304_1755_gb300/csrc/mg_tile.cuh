// Constant-coefficient V(1,1) level kernels, shared-memory tiled (included by k_mg.cu
// after mg_kernels.cuh).
//
// With c = omega / (8/3) and A = 3 I - S9/3 (S9 = 3 x 3 box sum) the fused level
// operations are separable filters:
//   down:  b_c = P^T (b - A c b) = (1 - 3c) (r3 (x) r3) b + (c/3) (r5 (x) r5) b,
//          r3 = (1/2, 1, 1/2), r5 = r3 * (1,1,1) = (1/2, 3/2, 2, 3/2, 1/2), centred on the
//          fine node 2I+1 that carries coarse node I;
//   up:    x = c b + e (e = P x_c) followed by one Jacobi step:
//          x' = (2c - 3c^2) b + (1 - 3c) e + S9 g,   g = (c^2/3) b + (c/3) e.
// A CTA first copies the window of the fine (and coarse) grid its tile needs into shared
// memory with 16-byte cp.async copies -- many bytes in flight per SM, which is what a
// streaming stencil needs to run at HBM speed -- and then evaluates the filters from
// shared memory, each warp walking a few rows with the partial sums in registers.
// Level arrays have an odd row length, so rows are not 16-byte aligned: the loader
// copies the aligned middle of every row segment asynchronously and the ragged ends with
// plain loads, and never reads outside the array.
#pragma once
#include <cstdint>
#include <type_traits>

namespace {
constexpr int MT_THREADS = 256;
constexpr int MD_TX = 64, MD_TY = 16;     // down: coarse tile (columns x rows)
constexpr int MU_FX = 128;                // up: fine tile columns; rows: mu_fy<TB, TS>()
// rows of the up tile: 32, or 16 for FP64 arithmetic (the two windows stay below 48 KB of shared
// memory; a thread recomputes two window rows per RW = rows / 4 output rows)
template <typename TB, typename TS, typename TA> constexpr int mu_fy() {
  return sizeof(TA) == 8 ? 16 : 32;
}

template <typename T> __device__ __forceinline__ T zero_of() { return T(0); }
template <> __device__ __forceinline__ bf16 zero_of<bf16>() { return __float2bfloat16_rn(0.f); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Shared-memory row pitch (elements) for a window NC columns wide: room for the
// alignment phase (< 16 bytes) and a multiple of 16 bytes.
template <typename T, int NC> constexpr int win_pitch() {
  constexpr int V = 16 / (int)sizeof(T);
  return ((NC + 2 * V - 2) / V) * V;
}

// Copies rows [r0, r0 + NR) x columns [c0, c0 + NC) of the m x m array g into sw (row rr at
// sw + rr * SW + sph[rr]), with zeros outside the array.  Call with all MT_THREADS threads,
// then cp_async_wait_all() and __syncthreads() before reading.  Each warp takes rows
// warp, warp + 8, ...: the 16-byte aligned middle of a row goes by cp.async, the up to
// 2 (V - 1) ragged end elements by plain loads that are all issued before any of them is
// stored, so a warp waits for one memory latency, not one per row.
template <typename T, int NR, int NC, bool OVER = false>
__device__ __forceinline__ void load_window(const T* __restrict__ g, int m, int r0, int c0, T* sw, int* sph) {
  constexpr int V = 16 / (int)sizeof(T);
  constexpr int SW = win_pitch<T, NC>();
  constexpr int NW = MT_THREADS / 32;
  constexpr int RPW = (NR + NW - 1) / NW;               // rows per warp
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (OVER) {
    // guarded array: copy whole aligned 16-byte chunks around every row segment; the bytes outside
    // the segment land in the row's slack or in columns fix_window_columns() zeroes afterwards
    for (int rr = warp; rr < NR; rr += NW) {
      const int r = r0 + rr;
      T* srow = sw + rr * SW;
      if (r < 0 || r >= m) {
        for (int k = lane; k < NC; k += 32) srow[k] = zero_of<T>();
        if (lane == 0) sph[rr] = 0;
        continue;
      }
      const uintptr_t a0 = (uintptr_t)(g + (size_t)r * m) + (uintptr_t)((intptr_t)c0 * (intptr_t)sizeof(T));
      const int ph = (int)((a0 & 15u) / sizeof(T));
      if (lane == 0) sph[rr] = ph;
      const char* src = (const char*)(a0 & ~(uintptr_t)15);
      const int nch = (ph + NC + V - 1) / V;            // <= NCH
      for (int q = lane; q < nch; q += 32) cp_async16((char*)srow + 16 * q, src + 16 * q);
    }
    return;
  }
  T endv[RPW];
  int endk[RPW];                                        // window column of this lane's end element, or -1
#pragma unroll
  for (int q = 0; q < RPW; ++q) {
    const int rr = warp + q * NW;
    endk[q] = -1;
    endv[q] = zero_of<T>();
    if (rr >= NR) continue;
    const int r = r0 + rr;
    if (r < 0 || r >= m) {
      if (lane == 0) sph[rr] = 0;
      continue;
    }
    const T* grow = g + (size_t)r * m;
    const uintptr_t a0 = (uintptr_t)grow + (uintptr_t)((intptr_t)c0 * (intptr_t)sizeof(T));
    const int ph = (int)((a0 & 15u) / sizeof(T));
    if (lane == 0) sph[rr] = ph;
    T* sbase = sw + rr * SW + ph;                       // column c0 + k lands at sbase[k]
    const int cl = max(c0, 0), cr = min(c0 + NC, m);
    const int ca = cl + (V - (cl - c0 + ph) % V) % V;   // first 16-byte aligned column >= cl
    const int nch = cr > ca ? (cr - ca) / V : 0;
    const int cb = ca + nch * V;
    for (int qq = lane; qq < nch; qq += 32) cp_async16(sbase + (ca - c0) + qq * V, grow + ca + qq * V);
    // ragged ends: [cl, min(ca, cr)) and [max(cb, ca), cr), at most V - 1 columns each
    const int nh = min(ca, cr) - cl, t0 = max(cb, ca), ntl = cr - t0;
    int c = -1;
    if (lane < V - 1) c = lane < nh ? cl + lane : -1;
    else if (lane < 2 * (V - 1)) c = lane - (V - 1) < ntl ? t0 + lane - (V - 1) : -1;
    if (c >= 0) {
      endv[q] = grow[c];
      endk[q] = c - c0;
    }
  }
#pragma unroll
  for (int q = 0; q < RPW; ++q) {
    const int rr = warp + q * NW;
    if (rr >= NR) continue;
    const int r = r0 + rr;
    T* srow = sw + rr * SW;
    if (r < 0 || r >= m) {
      for (int k = lane; k < NC; k += 32) srow[k] = zero_of<T>();
      continue;
    }
    const uintptr_t a0 = (uintptr_t)(g + (size_t)r * m) + (uintptr_t)((intptr_t)c0 * (intptr_t)sizeof(T));
    T* sbase = srow + (int)((a0 & 15u) / sizeof(T));
    if (endk[q] >= 0) sbase[endk[q]] = endv[q];
    // zeros left and right of the grid
    const int zl = max(0, min(NC, -c0)), zr = max(0, min(NC, c0 + NC - m));
    for (int k = lane; k < zl; k += 32) sbase[k] = zero_of<T>();
    for (int k = lane; k < zr; k += 32) sbase[NC - 1 - k] = zero_of<T>();
  }
}

// After an over-fetching load_window has landed and the CTA has synchronised: zero the window
// columns outside [0, m) (only tiles at the left or right edge of the grid have any) and
// synchronise again if anything was written.
template <typename T, int NR, int NC>
__device__ __forceinline__ void fix_window_columns(T* sw, const int* sph, int c0, int m) {
  constexpr int SW = win_pitch<T, NC>();
  if (c0 >= 0 && c0 + NC <= m) return;                  // uniform over the CTA
  const int zl = max(0, min(NC, -c0)), zr = max(0, min(NC, c0 + NC - m));
  for (int t = threadIdx.x; t < NR * 32; t += MT_THREADS) {
    const int rr = t >> 5, k = t & 31;
    T* sbase = sw + rr * SW + sph[rr];
    for (int q = k; q < zl; q += 32) sbase[q] = zero_of<T>();
    for (int q = k; q < zr; q += 32) sbase[NC - 1 - q] = zero_of<T>();
  }
  __syncthreads();
}

template <typename TA, typename T> __device__ __forceinline__ TA sld(const T* p) { return ld_as<TA>(p); }

// ---------------------------------------------------------------------------
// down: tile of MD_TX x MD_TY coarse nodes; fine window rows 2J0-1 .. 2J0+2MD_TY+1,
// columns 2I0-1 .. 2I0+2MD_TX+1.  Warp w: coarse columns 32 (w & 1) + lane, coarse rows
// 4 (w >> 1) .. +3.
// OB: b lies in a guarded array (load_window may over-fetch aligned chunks).
template <typename TB, typename TS, typename TA, bool OB = false>
__global__ void __launch_bounds__(MT_THREADS) mg_down_tile(const TB* __restrict__ b, TS* __restrict__ bc, int m,
                                                           int mc, size_t ldb, size_t ldc, TA c, int tiles_x) {
  constexpr int NR = 2 * MD_TY + 3, NC = 2 * MD_TX + 3, SW = win_pitch<TB, NC>();
  __shared__ __align__(16) TB sw[NR * SW];
  __shared__ int sph[NR];
  const int I0 = (blockIdx.x % tiles_x) * MD_TX, J0 = (blockIdx.x / tiles_x) * MD_TY;
  load_window<TB, NR, NC, OB>(b + (size_t)blockIdx.y * ldb, m, 2 * J0 - 1, 2 * I0 - 1, sw, sph);
  cp_async_wait_all();
  __syncthreads();
  if (OB) fix_window_columns<TB, NR, NC>(sw, sph, 2 * I0 - 1, m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = 32 * (warp & 1) + lane;           // coarse column within the tile
  const int jw = 4 * (warp >> 1);                 // first coarse row of this warp
  const int I = I0 + i;
  const TA a3 = TA(1) - TA(3) * c, a5 = c / TA(3);
  TA h3[11], h5[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) {
    const int rr = 2 * jw + k;
    const TB* row = sw + rr * SW + sph[rr] + 2 * i;     // window columns 2i .. 2i+4
    const TA x0 = sld<TA>(row), x1 = sld<TA>(row + 1), x2 = sld<TA>(row + 2), x3 = sld<TA>(row + 3),
             x4 = sld<TA>(row + 4);
    h3[k] = TA(0.5) * (x1 + x3) + x2;
    h5[k] = TA(0.5) * (x0 + x4) + TA(1.5) * (x1 + x3) + TA(2) * x2;
  }
  TS* cb = bc + (size_t)blockIdx.y * ldc;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int J = J0 + jw + q;
    const TA v3 = TA(0.5) * (h3[2 * q + 1] + h3[2 * q + 3]) + h3[2 * q + 2];
    const TA v5 = TA(0.5) * (h5[2 * q] + h5[2 * q + 4]) + TA(1.5) * (h5[2 * q + 1] + h5[2 * q + 3]) + TA(2) * h5[2 * q + 2];
    if (I < mc && J < mc) st_as<TS, TA>(cb + (size_t)J * mc + I, a3 * v3 + a5 * v5);
  }
}

// ---------------------------------------------------------------------------
// up: tile of MU_FX x MU_FY fine nodes starting at (X0, Y0) (both even).  The windows hold the fine
// nodes Y0-1 .. Y0+MU_FY (rows) x X0-1 .. X0+MU_FX (columns) of b and the coarse nodes around them;
// coarse window node (R, C) is fine window node (2R, 2C), so the bilinear prolongation e = P x_c at
// fine window node (r, c) is x_c itself for even r and c, the mean of the two coarse neighbours along
// an odd coordinate and of the four around it when both are odd.  No node needs a test: the windows
// are zero outside the grid, and a fine node outside it (or on its boundary) only interpolates coarse
// nodes outside it, so its b, e and g are zero.  The result is
// x' = (2c - 3c^2) b + (1 - 3c) e + S9 g = alpha g + beta b + S9 g,  g = (c^2/3) b + (c/3) e,
// alpha = (1 - 3c)/(c/3), beta = 2c - 3c^2 - alpha c^2/3.  Each thread owns two output columns and
// walks RW + 2 window rows upwards: per row it forms g at its four columns from b and the coarse
// row's horizontal interpolants (carried from one even row to the next), the two horizontal
// three-sums of g, and finishes the row below once the row above it is known -- one pass over the
// windows with the partial sums in registers.
// OB, OC: b, x_c lie in guarded arrays (load_window may over-fetch aligned chunks).
// zmax (FP32 output only, may be null): per block, the largest |x| written, as float bits, merged by
// atomicMax into zmax[block] (non-negative floats order like their bit patterns; a NaN wins).
template <typename TB, typename TS, typename TA, typename TO = TS, bool OB = false, bool OC = false>
__global__ void __launch_bounds__(MT_THREADS) mg_up_tile(const TB* __restrict__ b, const TS* __restrict__ xc,
                                                         TO* __restrict__ x, int m, int mc, size_t ldb, size_t ldc,
                                                         size_t ldx, TA c, int tiles_x, unsigned* zmax = nullptr) {
  constexpr int MU_FY = mu_fy<TB, TS, TA>(), RW = MU_FY / 4;   // tile rows, rows per thread
  constexpr int NRB = MU_FY + 2, NCB = MU_FX + 2, SWB = win_pitch<TB, NCB>();
  constexpr int NRC = MU_FY / 2 + 3, NCC = MU_FX / 2 + 3, SWC = win_pitch<TS, NCC>();
  static_assert(MU_FX == 128 && MT_THREADS == 256 && RW % 2 == 0, "two columns per thread, 64 threads per row band");
  __shared__ __align__(16) TB sb[NRB * SWB];
  __shared__ __align__(16) TS sc[NRC * SWC];
  __shared__ int phb[NRB], phc[NRC];
  const int X0 = (blockIdx.x % tiles_x) * MU_FX, Y0 = (blockIdx.x / tiles_x) * MU_FY;
  load_window<TB, NRB, NCB, OB>(b + (size_t)blockIdx.y * ldb, m, Y0 - 1, X0 - 1, sb, phb);
  load_window<TS, NRC, NCC, OC>(xc + (size_t)blockIdx.y * ldc, mc, Y0 / 2 - 1, X0 / 2 - 1, sc, phc);
  cp_async_wait_all();
  __syncthreads();
  if (OB) fix_window_columns<TB, NRB, NCB>(sb, phb, X0 - 1, m);
  if (OC) fix_window_columns<TS, NRC, NCC>(sc, phc, X0 / 2 - 1, mc);
  const TA cgb = c * c / TA(3), cge = c / TA(3), cbb = TA(2) * c - TA(3) * c * c, cee = TA(1) - TA(3) * c;
  const TA alpha = cee / cge, beta = cbb - alpha * cgb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = 64 * (warp & 1) + 2 * lane;                   // window columns k0 .. k0 + 3 (k0 even)
  const int jw = RW * (warp >> 1);                             // window rows jw .. jw + RW + 1 (jw even)
  const int C0 = k0 / 2;                                       // coarse window columns C0 .. C0 + 2
  // horizontal interpolants of coarse window row R at the fine window columns k0 .. k0 + 3
  auto hrow = [&](int R, TA* hv) {
    const TS* cr = sc + R * SWC + phc[R] + C0;
    const TA x0 = sld<TA>(cr), x1 = sld<TA>(cr + 1), x2 = sld<TA>(cr + 2);
    hv[0] = x0, hv[1] = TA(0.5) * (x0 + x1), hv[2] = x1, hv[3] = TA(0.5) * (x1 + x2);
  };
  TA hA[4];
  int R = jw / 2;
  hrow(R, hA);
  TA Hm2[2] = {0, 0}, Hm1[2] = {0, 0}, gm1[2] = {0, 0}, bm1[2] = {0, 0};
  const int i0 = X0 + k0, i1 = i0 + 1;                         // fine columns of the outputs
  TO* xb = x + (size_t)blockIdx.y * ldx;
  unsigned vmax = 0;                                           // |outputs| as float bits (FP32 output)
#pragma unroll
  for (int k = 0; k < RW + 2; ++k) {
    const int r = jw + k;
    TA e[4];
    if ((k & 1) == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) e[q] = hA[q];
    } else {
      TA hB[4];
      hrow(R + 1, hB);
#pragma unroll
      for (int q = 0; q < 4; ++q) e[q] = TA(0.5) * (hA[q] + hB[q]), hA[q] = hB[q];
      ++R;
    }
    const TB* br = sb + r * SWB + phb[r] + k0;
    TA bv[4], g[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) bv[q] = sld<TA>(br + q), g[q] = cgb * bv[q] + cge * e[q];
    const TA H0 = (g[0] + g[1]) + g[2], H1 = (g[1] + g[2]) + g[3];
    if (k >= 2) {                                               // window row r - 1 = fine row Y0 + r - 2
      const int j = Y0 + r - 2;
      if (j < m) {
        TO* op = xb + (size_t)j * m;
        const TA v0 = alpha * gm1[0] + beta * bm1[0] + ((Hm2[0] + Hm1[0]) + H0);
        const TA v1 = alpha * gm1[1] + beta * bm1[1] + ((Hm2[1] + Hm1[1]) + H1);
        if (i0 < m) st_as<TO, TA>(op + i0, v0);
        if (i1 < m) st_as<TO, TA>(op + i1, v1);
        if constexpr (std::is_same<TO, float>::value && std::is_same<TA, float>::value) {
          if (i0 < m) vmax = max(vmax, __float_as_uint(fabsf(v0)));
          if (i1 < m) vmax = max(vmax, __float_as_uint(fabsf(v1)));
        }
      }
    }
    Hm2[0] = Hm1[0], Hm2[1] = Hm1[1];
    Hm1[0] = H0, Hm1[1] = H1;
    gm1[0] = g[1], gm1[1] = g[2];
    bm1[0] = bv[1], bm1[1] = bv[2];
  }
  if constexpr (std::is_same<TO, float>::value && std::is_same<TA, float>::value) {
    if (zmax) {                                                // uniform over the grid
      __shared__ unsigned cmax;
      if (threadIdx.x == 0) cmax = 0;
      for (int o = 16; o > 0; o >>= 1) vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      __syncthreads();
      if (lane == 0 && vmax) atomicMax(&cmax, vmax);
      __syncthreads();
      if (threadIdx.x == 0 && cmax) atomicMax(zmax + blockIdx.y, cmax);
    }
  }
}
}  // namespace
