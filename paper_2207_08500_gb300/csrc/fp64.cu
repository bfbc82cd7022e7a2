// FP64 path of the NENO6 Euler right-hand side (Li, Fu & Adams, arXiv
// 2207.08500): one fused kernel per RHS evaluation (optionally with the SSP-RK3
// stage combination as its epilogue), the batched classifier, and the CFL
// reduction.
//
// Every binary64 operation is written with an explicit round-to-nearest
// intrinsic (__dadd_rn, __dmul_rn, __fma_rn, __ddiv_rn, __dsqrt_rn, ...) in the
// fixed order the scheme is specified in, so the compiler can neither contract
// nor reorder it; the classifier masks are therefore a deterministic function
// of the state, identical on any IEEE-754 implementation of that order.
//
// Design (GB300): binary64 arithmetic runs on the SM's FP64 pipe, and the
// classifier (3104 multiply-adds per call, 16 calls per cell and RHS) is ~97 %
// of the work, so this kernel is bound by that pipe.  Each CTA owns a tile of
// cells, stages the tile plus a 3-cell halo (periodic wrap or zero-gradient
// copy done in the load) and every per-cell quantity in shared memory once,
// then runs one work item per (face, characteristic field) with four lanes
// per face.  Classifier weights live in the kernel's parameter block
// (constant bank), so the multiply-adds take the weight as a constant operand
// and the warp reads it by broadcast.  Cheap comparisons (ReLU, max, |x|) are
// done on the integer pipe on the bit patterns to keep the FP64 pipe for the
// arithmetic.
#include "fp64_ops.cuh"
#include "internal.h"
#include "tc.cuh"

namespace neno6 {
namespace {

using namespace f64ops;

constexpr int kThreads = 256;

template <int NDIM>
struct Geom;
// Staged tile: TX x TY cells and a 3-cell halo; staged column bx holds
// global column i0 - X0 + bx.  In 2D the tile's rows are 40 cells wide
// (i0-4 .. i0+35) so that a TMA copy of the box can start on a 16-byte
// boundary (an even float64 column); the outer two columns are staged but
// never read.
template <>
struct Geom<2> {
  static constexpr int TX = 32, TY = 16, HY = 3, NV = 4;
  static constexpr int X0 = 4, SX = TX + 8, SY = TY + 6;
  static constexpr int NXF = TY * (TX + 1);  // x faces of a tile
  static constexpr int NYF = (TY + 1) * TX;  // y faces of a tile
};
template <>
struct Geom<1> {
  static constexpr int TX = 63, TY = 1, HY = 0, NV = 3;
  static constexpr int X0 = 3, SX = TX + 6, SY = 1;
  static constexpr int NXF = TX + 1;
  static constexpr int NYF = 0;
};

// Per-cell arrays staged in shared memory (structure of arrays).
template <int NV>
struct CellArrays {
  static constexpr int U = 0;                // NV conserved variables
  static constexpr int u = NV, v = NV + 1, c = NV + 2, H = NV + 3, s = NV + 4;
  static constexpr int Fx = NV + 5;          // NV x-fluxes
  static constexpr int Fy = Fx + NV;         // NV y-fluxes (2D)
  static constexpr int N = Fy + NV;
};

// Per-thread slot parked in shared memory while the classifier runs (keeps
// the stencils and the R row out of registers): "+" stencil, mirrored "-"
// stencil, R row.
constexpr int kPark = 16;

template <int NDIM>
constexpr size_t rhs_smem_bytes() {
  using G = Geom<NDIM>;
  // ... then one mbarrier (the tile's TMA copy)
  return sizeof(double) * (size_t(CellArrays<G::NV>::N) * G::SX * G::SY +
                           size_t(G::NV) * G::TY * (G::TX + 1) +
                           size_t(G::NV) * (G::TY + 1) * G::TX + size_t(kPark) * kThreads + 1);
}

// The 2D tile at (i0, j0) is copied by TMA: U described by the tensor map
// (in the parameter space, 64-byte aligned) and the whole staged box inside
// the grid (no periodic wrap, no clamp).  The box's first column i0 - 4 is
// even, hence 16-byte aligned.
__device__ __forceinline__ bool tile_by_tma(const RhsArgs& a, int i0, int j0) {
  using G = Geom<2>;
  return a.use_tma && (reinterpret_cast<uintptr_t>(&a.tmap) & 63u) == 0 && i0 - G::X0 >= 0 &&
         i0 - G::X0 + G::SX <= a.nx && j0 - G::HY >= 0 && j0 - G::HY + G::SY <= a.ny;
}

template <int NDIM>
__global__ void __launch_bounds__(kThreads, 1) rhs_fp64_kernel(const __grid_constant__ RhsParamsF64 P) {
  using G = Geom<NDIM>;
  using CA = CellArrays<G::NV>;
  constexpr int NV = G::NV, SX = G::SX, SY = G::SY, NC = SX * SY;
  constexpr int TX = G::TX, TY = G::TY;
  extern __shared__ __align__(1024) double smem[];
  double* C = smem;                        // [CA::N][NC]
  double* sFx = smem + CA::N * NC;         // [NV][TY][TX+1]
  double* sFy = sFx + NV * TY * (TX + 1);  // [NV][TY+1][TX]
  double* park = sFy + NV * (TY + 1) * TX + threadIdx.x;  // [kPark][kThreads]
  uint64_t* tbar = reinterpret_cast<uint64_t*>(sFy + NV * (TY + 1) * TX + kPark * kThreads);
  const RhsArgs& a = P.a;
  const double* __restrict__ net = P.net.p;
  const int nx = a.nx, ny = a.ny;
  const size_t plane = (size_t)nx * ny;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const double gm1 = a.gm1, gamma = a.gamma;

  // ---- 1. tile + halo and per-cell quantities.  An interior 2D tile's
  // conserved variables arrive by one TMA copy of the box [NV][SY][SX]
  // straight into the CA::U planes; edge tiles (ghost cells by periodic wrap
  // or zero-gradient clamp) and 1D tiles are loaded cell by cell.
  bool by_tma = false;
  if (NDIM == 2) {
    by_tma = tile_by_tma(a, i0, j0);
    if (by_tma) {
      if (threadIdx.x == 0) {
        tc::mbar_init(tbar, 1);
        tc::fence_mbar_init();
        tc::mbar_arrive_expect_tx(tbar, (uint32_t)(NV * NC * sizeof(double)));
        tc::tma_load_3d(C + CA::U * NC, &a.tmap, tbar, i0 - G::X0, j0 - G::HY, 0);
      }
      __syncthreads();  // the barrier is initialised before anyone waits on it
      const bool timed_out = !tc::mbar_wait(tbar, 0);
      if (__syncthreads_or(timed_out)) {
        // the copy may still be in flight: wait once more (bounded) before
        // the CTA's shared memory is released
        tc::mbar_wait(tbar, 0);
        if (threadIdx.x == 0) atomicOr(a.status, 4);
        return;
      }
    }
  }
  for (int e = threadIdx.x; e < NC; e += kThreads) {
    const int bx = e % SX, by = e / SX;
    double U[NV];
    if (by_tma) {
#pragma unroll
      for (int n = 0; n < NV; ++n) U[n] = C[(CA::U + n) * NC + e];
    } else {
      const int gi = wrap_index(i0 - G::X0 + bx, nx, a.bcx);
      const int gj = NDIM == 2 ? wrap_index(j0 - G::HY + by, ny, a.bcy) : 0;
      const size_t g = (size_t)gj * nx + gi;
#pragma unroll
      for (int n = 0; n < NV; ++n) {
        U[n] = a.U[n * plane + g];
        C[(CA::U + n) * NC + e] = U[n];
      }
    }
    const double rho = U[0], E = U[NV - 1];
    const double u = __ddiv_rn(U[1], rho);
    double v = 0.0, q;
    if (NDIM == 2) {
      v = __ddiv_rn(U[2], rho);
      q = __fma_rn(v, v, __dmul_rn(u, u));
    } else {
      q = __dmul_rn(u, u);
    }
    const double p = __dmul_rn(gm1, __dsub_rn(E, __dmul_rn(0.5, __dmul_rn(rho, q))));
    const double c = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), rho));
    const double Ep = __dadd_rn(E, p);
    if (!(rho > 0.0) || !(p > 0.0)) atomicOr(a.status, 1);
    C[CA::u * NC + e] = u;
    C[CA::v * NC + e] = v;
    C[CA::c * NC + e] = c;
    C[CA::H * NC + e] = __ddiv_rn(Ep, rho);
    C[CA::s * NC + e] = __dsqrt_rn(rho);
    if (NDIM == 2) {
      C[(CA::Fx + 0) * NC + e] = U[1];
      C[(CA::Fx + 1) * NC + e] = __fma_rn(U[1], u, p);
      C[(CA::Fx + 2) * NC + e] = __dmul_rn(U[2], u);
      C[(CA::Fx + 3) * NC + e] = __dmul_rn(Ep, u);
      C[(CA::Fy + 0) * NC + e] = U[2];
      C[(CA::Fy + 1) * NC + e] = __dmul_rn(U[1], v);
      C[(CA::Fy + 2) * NC + e] = __fma_rn(U[2], v, p);
      C[(CA::Fy + 3) * NC + e] = __dmul_rn(Ep, v);
    } else {
      C[(CA::Fx + 0) * NC + e] = U[1];
      C[(CA::Fx + 1) * NC + e] = __fma_rn(U[1], u, p);
      C[(CA::Fx + 2) * NC + e] = __dmul_rn(Ep, u);
    }
  }

  // dt of an RK3 step (stage 1 computes it from max(|u|+c), max(|v|+c)).
  double dt = 0.0;
  if (a.stage == 1) {
    const double sx = __longlong_as_double((long long)a.smax[0]);
    double s = __ddiv_rn(sx, a.dx);
    if (NDIM == 2) s = __dadd_rn(s, __ddiv_rn(__longlong_as_double((long long)a.smax[1]), a.dy));
    dt = __ddiv_rn(a.cfl, s);
    const double t = *a.t_dev;
    if (a.t_end > 0.0 && __dadd_rn(t, dt) > a.t_end) dt = __dsub_rn(a.t_end, t);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
      *a.dt_dev = dt;
      if (a.dt_user) *a.dt_user = dt;
    }
  } else if (a.stage >= 2) {
    dt = *a.dt_dev;
    if (a.stage == 3 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
      *a.t_dev = __dadd_rn(*a.t_dev, dt);
  }
  __syncthreads();

  // ---- 2. faces: one item per (face, field), four lanes per face
  constexpr int NITEMS = 4 * (G::NXF + G::NYF);
  static_assert((4 * G::NXF) % 32 == 0, "x/y items must not share a warp");
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int base = 0; base < NITEMS; base += kThreads) {
    const int w = base + threadIdx.x;
    if (base + (threadIdx.x & ~31) >= NITEMS) break;  // whole warp past the end
    const int face = w >> 2;
    const int m = min(w & 3, NV - 1);
    const int dir = face < G::NXF ? 0 : 1;  // warp-uniform
    int cb0, stride, gf, gline;
    if (dir == 0) {
      const int r = face / (TX + 1), f = face % (TX + 1);
      cb0 = (G::HY + r) * SX + (G::X0 - 3) + f;
      stride = 1;
      gf = i0 + f;      // global face index along x, 0..nx
      gline = j0 + r;   // row
    } else {
      const int fl = face - G::NXF;
      const int f = fl / TX, c = fl % TX;
      cb0 = f * SX + G::X0 + c;
      stride = SX;
      gf = j0 + f;
      gline = i0 + c;   // column
    }
    const bool valid = (w & 3) < NV &&
                       (dir == 0 ? (gf <= nx && gline < ny) : (gf <= ny && gline < nx));
    const double* Fl = C + (dir == 0 ? CA::Fx : CA::Fy) * NC;
    const double* Un = C + (dir == 0 ? CA::u : CA::v) * NC;  // normal velocity
    const int ca = cb0 + 2 * stride, cbb = cb0 + 3 * stride;

    // Roe average of cells i and i+1 (Sec. 4.4).
    const double sa = C[CA::s * NC + ca], sb = C[CA::s * NC + cbb];
    const double den = __dadd_rn(sa, sb);
    const double ut = __ddiv_rn(__fma_rn(sb, C[CA::u * NC + cbb], __dmul_rn(sa, C[CA::u * NC + ca])), den);
    const double Ht = __ddiv_rn(__fma_rn(sb, C[CA::H * NC + cbb], __dmul_rn(sa, C[CA::H * NC + ca])), den);
    double vt = 0.0, qt;
    if (NDIM == 2) {
      vt = __ddiv_rn(__fma_rn(sb, C[CA::v * NC + cbb], __dmul_rn(sa, C[CA::v * NC + ca])), den);
      qt = __fma_rn(vt, vt, __dmul_rn(ut, ut));
    } else {
      qt = __dmul_rn(ut, ut);
    }
    const double c2 = __dmul_rn(gm1, __dsub_rn(Ht, __dmul_rn(0.5, qt)));
    if (valid && !(c2 > 0.0)) atomicOr(a.status, 2);
    const double ct = __dsqrt_rn(c2);
    const double ic = __ddiv_rn(1.0, ct);
    const double b1 = __ddiv_rn(gm1, c2);
    const double b2 = __dmul_rn(0.5, __dmul_rn(b1, qt));
    const double nt = dir == 0 ? ut : vt;
    const double nc = __dmul_rn(nt, ic);
    const double b1u = __dmul_rn(b1, ut), b1v = __dmul_rn(b1, vt);
    const double hb1 = __dmul_rn(0.5, b1), ntc = __dmul_rn(nt, ct);

    // Left eigenvector (row m of L) and right-eigenvector components (row m
    // of R, i.e. component m of every column) in the Roe/Toro scaling.
    double L[4], R[4];
    {
      const double am = __dmul_rn(0.5, __dadd_rn(b2, nc));   // acoustic "-" first entry
      const double ap = __dmul_rn(0.5, __dsub_rn(b2, nc));   // acoustic "+" first entry
      const double nb1u = -b1u, nb1v = -b1v;
      const double hm_u = __dmul_rn(0.5, __dsub_rn(nb1u, ic)), hp_u = __dmul_rn(0.5, __dadd_rn(nb1u, ic));
      if (NDIM == 1) {
        if (m == 0) { L[0] = am; L[1] = hm_u; L[2] = hb1; }
        else if (m == 1) { L[0] = __dsub_rn(1.0, b2); L[1] = b1u; L[2] = -b1; }
        else { L[0] = ap; L[1] = hp_u; L[2] = hb1; }
        L[3] = 0.0;
        if (m == 0) { R[0] = 1.0; R[1] = 1.0; R[2] = 1.0; }
        else if (m == 1) { R[0] = __dsub_rn(ut, ct); R[1] = ut; R[2] = __dadd_rn(ut, ct); }
        else { R[0] = __dsub_rn(Ht, ntc); R[1] = __dmul_rn(0.5, qt); R[2] = __dadd_rn(Ht, ntc); }
        R[3] = 0.0;
      } else {
        const double hnb1v = __dmul_rn(0.5, nb1v), hnb1u = __dmul_rn(0.5, nb1u);
        const double hm_v = __dmul_rn(0.5, __dsub_rn(nb1v, ic)), hp_v = __dmul_rn(0.5, __dadd_rn(nb1v, ic));
        if (m == 0) {
          L[0] = am; L[1] = dir == 0 ? hm_u : hnb1u; L[2] = dir == 0 ? hnb1v : hm_v; L[3] = hb1;
        } else if (m == 1) {
          L[0] = __dsub_rn(1.0, b2); L[1] = b1u; L[2] = b1v; L[3] = -b1;
        } else if (m == 2) {
          L[0] = dir == 0 ? -vt : -ut; L[1] = dir == 0 ? 0.0 : 1.0; L[2] = dir == 0 ? 1.0 : 0.0; L[3] = 0.0;
        } else {
          L[0] = ap; L[1] = dir == 0 ? hp_u : hnb1u; L[2] = dir == 0 ? hnb1v : hp_v; L[3] = hb1;
        }
        if (m == 0) { R[0] = 1.0; R[1] = 1.0; R[2] = 0.0; R[3] = 1.0; }
        else if (m == 1) {
          if (dir == 0) { R[0] = __dsub_rn(ut, ct); R[1] = ut; R[2] = 0.0; R[3] = __dadd_rn(ut, ct); }
          else { R[0] = ut; R[1] = ut; R[2] = 1.0; R[3] = ut; }
        } else if (m == 2) {
          if (dir == 0) { R[0] = vt; R[1] = vt; R[2] = 1.0; R[3] = vt; }
          else { R[0] = __dsub_rn(vt, ct); R[1] = vt; R[2] = 0.0; R[3] = __dadd_rn(vt, ct); }
        } else {
          R[0] = __dsub_rn(Ht, ntc); R[1] = __dmul_rn(0.5, qt); R[2] = dir == 0 ? vt : ut;
          R[3] = __dadd_rn(Ht, ntc);
        }
      }
    }

    // LLF alpha_m: max over the six stencil cells of |lambda_m|.
    double alpha = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int cj = cb0 + j * stride;
      const double un = Un[cj], cs = C[CA::c * NC + cj];
      const double lam = m == 0 ? __dsub_rn(un, cs) : (m == NV - 1 ? __dadd_rn(un, cs) : un);
      alpha = j == 0 ? dabs(lam) : dmax_nn(alpha, dabs(lam));
    }

    // Characteristic projection and LLF split of the six stencil cells.
    double sp[6], sm[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int cj = cb0 + j * stride;
      double vv = __dmul_rn(L[0], C[(CA::U + 0) * NC + cj]);
      double gg = __dmul_rn(L[0], Fl[0 * NC + cj]);
#pragma unroll
      for (int n = 1; n < NV; ++n) {
        vv = __fma_rn(L[n], C[(CA::U + n) * NC + cj], vv);
        gg = __fma_rn(L[n], Fl[n * NC + cj], gg);
      }
      sp[j] = __dmul_rn(0.5, __fma_rn(alpha, vv, gg));
      sm[j] = __dmul_rn(0.5, __fma_rn(-alpha, vv, gg));
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      park[j * kThreads] = sp[j];
      park[(6 + j) * kThreads] = sm[5 - j];  // the "-" side is the mirror image
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) park[(12 + q) * kThreads] = R[q];

    // Classifier bits of both sides ("-" side = mirror image).
    // Compiler-level barrier: the parked values must be re-read from shared
    // memory, not kept live in registers across the classifier.
    asm volatile("" ::: "memory");
    unsigned eta_side[2];
    if (a.mask_mode == kMaskMLP) {
#pragma unroll 1
      for (int side = 0; side < 2; ++side) {
        double st[6], x[6], z[4];
#pragma unroll
        for (int j = 0; j < 6; ++j) st[j] = park[(side * 6 + j) * kThreads];
        normalise6(st, x);
        eta_side[side] = mlp64(net, x, z);
      }
    } else if (a.mask_mode == kMaskTeno) {
      // TENO6-opt selection on the split fluxes themselves (its indicator
      // ratios do not depend on the scale)
#pragma unroll 1
      for (int side = 0; side < 2; ++side) {
        double st[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) st[j] = park[(side * 6 + j) * kThreads];
        eta_side[side] = teno6_eta(a.teno, st);
      }
    } else if (a.mask_mode == kMaskGiven) {
      size_t idx;
      if (dir == 0) idx = ((size_t)m * ny + gline) * (nx + 1) + gf;
      else idx = (size_t)NV * ny * (nx + 1) + ((size_t)m * (ny + 1) + gf) * nx + gline;
      const unsigned b = valid ? a.mask_in[idx] : 0u;
      eta_side[0] = b & 15u;
      eta_side[1] = b >> 4;
    } else {
      eta_side[0] = eta_side[1] = a.mask_mode == kMaskRough ? 15u : 0u;
    }
    asm volatile("" ::: "memory");
    double spl[6], smir[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      spl[j] = park[j * kThreads];
      smir[j] = park[(6 + j) * kThreads];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) R[q] = park[(12 + q) * kThreads];
    const double gp = combine64(a, spl, eta_side[0]);
    const double gmn = combine64(a, smir, eta_side[1]);
    const double gh = __dadd_rn(gp, gmn);

    // Back-projection F_n = sum_m R[n][m] gh_m; lane m of the face holds gh_m
    // and computes component n = m.
    const int fbase = lane & ~3;
    double ghm[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) ghm[q] = __shfl_sync(0xffffffffu, gh, fbase + q);
    double Fh = __dmul_rn(R[0], ghm[0]);
#pragma unroll
    for (int q = 1; q < NV; ++q) Fh = __fma_rn(R[q], ghm[q], Fh);

    if (valid) {
      if (dir == 0) {
        const int r = face / (TX + 1), f = face % (TX + 1);
        sFx[(m * TY + r) * (TX + 1) + f] = Fh;
      } else {
        const int fl = face - G::NXF;
        sFy[(m * (TY + 1) + fl / TX) * TX + fl % TX] = Fh;
      }
      if (a.mask_out) {
        size_t idx;
        if (dir == 0) idx = ((size_t)m * ny + gline) * (nx + 1) + gf;
        else idx = (size_t)NV * ny * (nx + 1) + ((size_t)m * (ny + 1) + gf) * nx + gline;
        a.mask_out[idx] = (uint8_t)(eta_side[0] | (eta_side[1] << 4));
      }
    }
  }
  __syncthreads();

  // ---- 3. conservative difference and (optionally) the RK3 stage update
  for (int e = threadIdx.x; e < TX * TY; e += kThreads) {
    const int c = e % TX, r = e / TX;
    const int gi = i0 + c, gj = j0 + r;
    if (gi >= nx || gj >= ny) continue;
    const size_t g = (size_t)gj * nx + gi;
    const int bc = (G::HY + r) * SX + G::X0 + c;
#pragma unroll
    for (int n = 0; n < NV; ++n) {
      const double Fp = sFx[(n * TY + r) * (TX + 1) + c + 1];
      const double Fm = sFx[(n * TY + r) * (TX + 1) + c];
      double rr = -__ddiv_rn(__dsub_rn(Fp, Fm), a.dx);
      if (NDIM == 2) {
        const double Gp = sFy[(n * (TY + 1) + r + 1) * TX + c];
        const double Gm = sFy[(n * (TY + 1) + r) * TX + c];
        rr = __dsub_rn(rr, __ddiv_rn(__dsub_rn(Gp, Gm), a.dy));
      }
      double val = rr;
      const double Ucur = C[(CA::U + n) * NC + bc];
      if (a.stage == 1) {
        val = __fma_rn(dt, rr, Ucur);
      } else if (a.stage == 2) {
        val = __fma_rn(0.75, a.U0[n * plane + g], __dmul_rn(0.25, __fma_rn(dt, rr, Ucur)));
      } else if (a.stage == 3) {
        val = __fma_rn(a.third, a.U0[n * plane + g], __dmul_rn(a.two_thirds, __fma_rn(dt, rr, Ucur)));
      }
      a.out[n * plane + g] = val;
    }
  }
}

__global__ void __launch_bounds__(256) classify_fp64_kernel(const __grid_constant__ ClassifyParamsF64 P) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P.n) return;
  double s[6], x[6], z[4];
#pragma unroll
  for (int j = 0; j < 6; ++j) s[j] = P.X[r * 6 + j];
  normalise6(s, x);
  const unsigned eta = mlp64(P.net.p, x, z);
  P.eta[r] = (uint8_t)eta;
  if (P.logits) {
#pragma unroll
    for (int k = 0; k < 4; ++k) P.logits[r * 4 + k] = z[k];
  }
}

// The same for the 6-32-32-32-4 network of the width study.
__global__ void __launch_bounds__(256) classify_fp64_narrow_kernel(const __grid_constant__ ClassifyParamsF64 P) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P.n) return;
  double s[6], x[6], z[4];
#pragma unroll
  for (int j = 0; j < 6; ++j) s[j] = P.X[r * 6 + j];
  normalise6(s, x);
  const unsigned eta = mlp64_narrow(P.net.p, x, z);
  P.eta[r] = (uint8_t)eta;
  if (P.logits) {
#pragma unroll
    for (int k = 0; k < 4; ++k) P.logits[r * 4 + k] = z[k];
  }
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// max over cells of |u|+c (and |v|+c): bit patterns of non-negative doubles
// order like the values, so integer max / atomicMax give the exact maximum.
template <int NDIM>
__global__ void __launch_bounds__(256) cfl_reduce_kernel(const double* __restrict__ U, int nx, int ny,
                                                         double gamma, unsigned long long* smax,
                                                         int* status) {
  const size_t plane = (size_t)nx * ny;
  const double gm1 = __dsub_rn(gamma, 1.0);
  unsigned long long mx = 0, my = 0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < plane;
       k += (size_t)gridDim.x * blockDim.x) {
    const double rho = U[k];
    const double E = U[(NDIM == 2 ? 3 : 2) * plane + k];
    const double u = __ddiv_rn(U[plane + k], rho);
    double v = 0.0, q;
    if (NDIM == 2) {
      v = __ddiv_rn(U[2 * plane + k], rho);
      q = __fma_rn(v, v, __dmul_rn(u, u));
    } else {
      q = __dmul_rn(u, u);
    }
    const double p = __dmul_rn(gm1, __dsub_rn(E, __dmul_rn(0.5, __dmul_rn(rho, q))));
    const double c = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), rho));
    if (!(rho > 0.0) || !(p > 0.0)) atomicOr(status, 1);
    mx = umax64(mx, (unsigned long long)dbits(__dadd_rn(dabs(u), c)));
    if (NDIM == 2) my = umax64(my, (unsigned long long)dbits(__dadd_rn(dabs(v), c)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = umax64(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    my = umax64(my, __shfl_xor_sync(0xffffffffu, my, o));
  }
  __shared__ unsigned long long wx[8], wy[8];
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    wx[warp] = mx;
    wy[warp] = my;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      mx = umax64(mx, wx[i]);
      my = umax64(my, wy[i]);
    }
    atomicMax(&smax[0], mx);
    if (NDIM == 2) atomicMax(&smax[1], my);
  }
}

}  // namespace

namespace {

// cuTensorMapEncodeTiled, reached through the runtime's driver entry-point
// query (the library links no driver library); null if unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// Tensor map of the 2D state U ([4][ny][nx] float64) with the box of one
// staged FP64 tile ([4][SY][SX]).  False when U cannot be described: the
// row stride nx * 8 and the base must be multiples of 16 bytes.
bool encode_tile_map(RhsArgs& a) {
  using G = Geom<2>;
  EncodeTiledFn enc = encode_tiled();
  if (!enc || a.nx % 2 != 0 || (reinterpret_cast<uintptr_t>(a.U) & 15u) != 0) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny, (cuuint64_t)G::NV};
  const cuuint64_t strides[2] = {(cuuint64_t)a.nx * 8, (cuuint64_t)a.nx * a.ny * 8};
  const cuuint32_t box[3] = {(cuuint32_t)G::SX, (cuuint32_t)G::SY, (cuuint32_t)G::NV};
  const cuuint32_t unit[3] = {1, 1, 1};
  return enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double*>(a.U), dims, strides, box, unit,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_rhs_fp64(int ndim, RhsParamsF64& p, cudaStream_t s) {
  p.a.use_tma = ndim == 2 && encode_tile_map(p.a) ? 1 : 0;
  if (ndim == 2) {
    using G = Geom<2>;
    constexpr size_t sm = rhs_smem_bytes<2>();
    cudaError_t e = cudaFuncSetAttribute(rhs_fp64_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((p.a.nx + G::TX - 1) / G::TX, (p.a.ny + G::TY - 1) / G::TY);
    rhs_fp64_kernel<2><<<grid, kThreads, sm, s>>>(p);
  } else {
    using G = Geom<1>;
    constexpr size_t sm = rhs_smem_bytes<1>();
    cudaError_t e = cudaFuncSetAttribute(rhs_fp64_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((p.a.nx + G::TX - 1) / G::TX, 1);
    rhs_fp64_kernel<1><<<grid, kThreads, sm, s>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_classify_fp64(const ClassifyParamsF64& p, bool narrow, cudaStream_t s) {
  if (p.n == 0) return cudaSuccess;
  const long long blocks = (p.n + 255) / 256;
  if (narrow)
    classify_fp64_narrow_kernel<<<(unsigned)blocks, 256, 0, s>>>(p);
  else
    classify_fp64_kernel<<<(unsigned)blocks, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_cfl_reduce(int ndim, const double* U, int nx, int ny, double gamma,
                              unsigned long long* smax, int* status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(smax, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const size_t cells = (size_t)nx * ny;
  unsigned blocks = (unsigned)((cells + 255) / 256);
  if (blocks > 152u * 8u) blocks = 152u * 8u;
  if (ndim == 2)
    cfl_reduce_kernel<2><<<blocks, 256, 0, s>>>(U, nx, ny, gamma, smax, status);
  else
    cfl_reduce_kernel<1><<<blocks, 256, 0, s>>>(U, nx, ny, gamma, smax, status);
  return cudaGetLastError();
}

}  // namespace neno6
