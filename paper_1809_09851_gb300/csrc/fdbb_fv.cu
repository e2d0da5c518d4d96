// fdbb_fv.cu -- batched explicit finite-volume steps (first-order Rusanov /
// local Lax-Friedrichs) on many periodic n^3 grids in one persistent launch.
//
// Each grid occupies a range of a "virtual" cell index space, padded to a
// multiple of FDBB_FV_TILE cells, so that a block-sized tile of virtual cells
// always belongs to one grid.  The grid table (up to FDBB_FV_MAX_GRIDS
// descriptors) travels in the kernel's parameter block.  The step kernels
// march 32 x 8-cell column tiles along z through shared-memory plane tiles and
// form the face fluxes from the paper's inviscid flux (section 2.2):
// k_fv_rusanov_step one plane at a time (FP64 grids), k_fv_rusanov_step2 two
// planes at a time in packed FP32x2 arithmetic (FP32 grids).  The time step
// of every grid comes from a per-grid maximum wave speed kept in a
// caller-provided scratch array of three slots per grid:
//   step s reads slot s%3 (max of the state at its start), reduces the new
//   state's wave speed into slot (s+1)%3 with atomicMax, and clears slot
//   (s+2)%3, which step s-1 read and step s+1 will fill.
// The maximum is order independent, so a grid's results do not depend on
// which other grids share the launch.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "fdbb.h"
#include "fdbb_device.cuh"
#include "fdbb_internal.h"

namespace fdbb {
namespace {

constexpr int kFvThreads = FDBB_FV_TILE;

// Tiles of the step kernel: a 32 x 8 (x, y) column segment of up to zseg
// planes (FvArgs::zseg, chosen per launch by fv_plan).
constexpr int kBX = 32, kBY = 8;
constexpr int kSX = kBX + 2, kSY = kBY + 2, kSlots = kSX * kSY;  // plane tile with a one-cell halo
constexpr int kSlotVals = 8;  // U[5], p, 1/rho, c

struct FvArgs {
  int ngrids;
  int zseg;          // step kernel: planes per column segment (even)
  int64_t vcells;    // virtual cells (sum of padded grid sizes)
  double gamma, cfl;
  void* smax;        // 3 slots per grid, storage type T
  unsigned long long* dbg;  // debug builds: index-check counters; else NULL
  int64_t tiles;     // step kernel: total tiles
  fdbb_fv_grid g[FDBB_FV_MAX_GRIDS];
  int64_t tile_begin[FDBB_FV_MAX_GRIDS];  // step kernel: first tile of each grid
};

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Host: tile table of the step kernel.
void fv_tiles(FvArgs& a) {
  int64_t t = 0;
  for (int i = 0; i < a.ngrids; ++i) {
    const int n = a.g[i].n;
    a.tile_begin[i] = t;
    t += (int64_t)ceil_div(n, kBX) * ceil_div(n, kBY) * ceil_div(n, a.zseg);
  }
  a.tiles = t;
}

// Grid owning step tile vt (tile_begin is sorted).
__device__ __forceinline__ int find_tile_grid(const FvArgs& a, int64_t vt) {
  int lo = 0, hi = a.ngrids - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.tile_begin[mid] <= vt) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Grid owning virtual cell vc: the last descriptor with cell_begin <= vc
// (descriptors are sorted by cell_begin).
__device__ __forceinline__ int find_grid(const FvArgs& a, int64_t vc) {
  int lo = 0, hi = a.ngrids - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.g[mid].cell_begin <= vc) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class T> __device__ __forceinline__ T ldg(const void* p, int64_t i) {
  return __ldg(static_cast<const T*>(p) + i);
}
// Load element i of a plane of `size` cells (debug builds: checked; an index
// out of range is recorded and reads 1).
template <class T>
__device__ __forceinline__ T ldg_in(unsigned long long* dbg, const void* p, int64_t i, int64_t size) {
  if (!FDBB_IDX_OK(dbg, i >= 0 && i < size, i)) return T(1);
  return ldg<T>(p, i);
}
// Store element i of a plane of `size` cells (debug builds: checked; an index
// out of range is recorded and skipped).
template <class T>
__device__ __forceinline__ void st_in(unsigned long long* dbg, void* p, int64_t i, int64_t size, T v) {
  if (!FDBB_IDX_OK(dbg, i >= 0 && i < size, i)) return;
  static_cast<T*>(p)[i] = v;
}

// Positive floating-point values order like their bit patterns.
__device__ __forceinline__ void atomic_max_pos(float* p, float v) {
  atomicMax(reinterpret_cast<int*>(p), __float_as_int(v));
}
__device__ __forceinline__ void atomic_max_pos(double* p, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(__double_as_longlong(v)));
}
__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <class T> __device__ __forceinline__ Consts<T> fv_consts(double g) {
  const double a1 = g - 1.0;
  return {T(g), T(a1), T(3.0 - g), T(2.0 / a1), T(1.0 / a1), T(-g)};
}

// Derived state for the finite-volume kernels.  FP64 grids use the IEEE
// derivation of the point-wise blocks.  FP32 grids use the hardware
// reciprocal and square-root approximations (relative error ~2^-22) and a
// plain internal-energy difference: the serving flows are smooth and
// subsonic, and the FP32 state's tolerance against the FP64 oracle is 2e-5.
__device__ __forceinline__ float fv_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float fv_sqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double fv_sqrt(double x) { return sqrt(x); }

__device__ __forceinline__ void fv_derive(Pt<double, 3>& s, const Consts<double>& k) {
  NoGuard g;
  derive(s, k, g);
}
// FP32 grids: 1/rho, p = (gamma - 1) (rhoE - |m|^2 / (2 rho)) and c^2 in the
// packed step kernel's sequence for one lane (derive2), so that the wave-speed
// maximum reduced from a state here and the one the step kernel reduces agree
// bit for bit.
__device__ __forceinline__ void fv_derive(Pt<float, 3>& s, const Consts<float>& k) {
  s.r = fv_rcp(s.rho);
  const float m2 = fmaf(s.m[2], s.m[2], fmaf(s.m[1], s.m[1], __fmul_rn(s.m[0], s.m[0])));
  s.p = __fmul_rn(k.a1, __fsub_rn(s.rE, __fmul_rn(0.5f, __fmul_rn(m2, s.r))));
  s.c2 = __fmul_rn(__fmul_rn(k.g, s.p), s.r);
}

// Derived state of the cell at linear index c of the planes P.
template <class T>
__device__ __forceinline__ void cell_state(void* const* P, int64_t c, const Consts<T>& k, Pt<T, 3>& s) {
  s.rho = ldg<T>(P[0], c);
  s.m[0] = ldg<T>(P[1], c);
  s.m[1] = ldg<T>(P[2], c);
  s.m[2] = ldg<T>(P[3], c);
  s.rE = ldg<T>(P[4], c);
  fv_derive(s, k);
}

template <class T> __device__ __forceinline__ T wave_speed_sum(const Pt<T, 3>& s) {
  const T c = fv_sqrt(s.c2);
  return (abs_(s.v[0]) + c) + (abs_(s.v[1]) + c) + (abs_(s.v[2]) + c);
}
// FP32: the sum as the packed step kernel forms it, (|m_x| + |m_y| + |m_z|) / rho + 3 c
__device__ __forceinline__ float wave_speed_sum(const Pt<float, 3>& s) {
  const float c = fv_sqrt(s.c2);
  return fmaf(__fadd_rn(__fadd_rn(fabsf(s.m[0]), fabsf(s.m[1])), fabsf(s.m[2])), s.r, __fmul_rn(3.0f, c));
}

template <class T> __global__ void __launch_bounds__(kFvThreads) k_fv_max_speed(const __grid_constant__ FvArgs a) {
  __shared__ int s_grid;
  const Consts<T> k = fv_consts<T>(a.gamma);
  for (int64_t base = (int64_t)blockIdx.x * kFvThreads; base < a.vcells; base += (int64_t)gridDim.x * kFvThreads) {
    if (threadIdx.x == 0) s_grid = find_grid(a, base);
    __syncthreads();
    const fdbb_fv_grid& g = a.g[s_grid];
    __syncthreads();
    const int64_t n = g.n, ncell = n * n * n;
    const int64_t c = base + threadIdx.x - g.cell_begin;
    T v = T(0);
    if (c >= 0 && c < ncell) {
      Pt<T, 3> s;
      cell_state<T>(g.U, c, k, s);
      v = wave_speed_sum(s);
    }
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0 && v > T(0)) atomic_max_pos(static_cast<T*>(a.smax) + 3 * g.slot + g.phase, v);
  }
}

// Shared-memory plane of a step tile: kSlotVals values for each of the kSlots
// cells of a (32+2) x (8+2) plane tile, structure of arrays.
template <class T> struct PlaneTile {
  T v[kSlotVals][kSlots];
};

// State, pressure, 1/rho and speed of sound of a cell given its conservative
// values u, into slot `slot` of plane tile P (each computed once per cell;
// the faces form the flux columns from them, which keeps the shared-memory
// traffic per cell at 8 values written and about 6 x 8 read).
template <class T>
__device__ __forceinline__ void put_slot(const T (&u)[5], const Consts<T>& k, PlaneTile<T>& P, int slot) {
  Pt<T, 3> s;
  s.rho = u[0];
  s.m[0] = u[1];
  s.m[1] = u[2];
  s.m[2] = u[3];
  s.rE = u[4];
  fv_derive(s, k);
#pragma unroll
  for (int q = 0; q < 5; ++q) P.v[q][slot] = u[q];
  P.v[5][slot] = s.p;
  P.v[6][slot] = s.r;
  P.v[7][slot] = fv_sqrt(s.c2);
}

template <class T>
__device__ __forceinline__ void load_cell(const FvArgs& a, const fdbb_fv_grid& g, int x, int y, int z, T (&u)[5]) {
  const int64_t c = ((int64_t)z * g.n + y) * g.n + x;
  const int64_t size = (int64_t)g.n * g.n * g.n;
#pragma unroll
  for (int q = 0; q < 5; ++q) u[q] = ldg_in<T>(a.dbg, g.U[q], c, size);
}

// Conservative values of this thread's (at most two) slots of one plane tile.
constexpr int kSlotsPerThread = (kSlots + kFvThreads - 1) / kFvThreads;
template <class T> struct SlotRaw {
  T u[kSlotsPerThread][5];
};

// One cell of a plane tile: U, p, 1/rho and c.
template <class T> struct Cell {
  T u[5], p, r, c;
};
template <class T> __device__ __forceinline__ Cell<T> cell_at(const PlaneTile<T>& P, int slot) {
  Cell<T> x;
#pragma unroll
  for (int q = 0; q < 5; ++q) x.u[q] = P.v[q][slot];
  x.p = P.v[5][slot];
  x.r = P.v[6][slot];
  x.c = P.v[7][slot];
  return x;
}

// What a face needs from one side in direction d: U, F_d(U) (the paper's
// inviscid flux column, section 2.2, with v = m / rho) and |v_d| + c.
template <class T> struct Side {
  T u[5], f[5], s;
};
template <class T, int d> __device__ __forceinline__ Side<T> side(const Cell<T>& e) {
  Side<T> x;
  const T md = e.u[1 + d];
#pragma unroll
  for (int q = 0; q < 5; ++q) x.u[q] = e.u[q];
  x.f[0] = md;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T vi = e.u[1 + i] * e.r;
    x.f[1 + i] = i == d ? fma_(md, vi, e.p) : md * vi;
  }
  const T vd = md * e.r;
  x.f[4] = vd * (e.u[4] + e.p);
  x.s = abs_(vd) + e.c;
  return x;
}
template <class T, int d> __device__ __forceinline__ Side<T> side(const PlaneTile<T>& P, int slot) {
  return side<T, d>(cell_at(P, slot));
}

// Twice the Rusanov flux through the face between the left side L and the
// right side R, (F(U_L) + F(U_R)) - s (U_R - U_L); the factor 1/2 is applied
// once per cell, to the sum of its face differences.
template <class T>
__device__ __forceinline__ void face(const Side<T>& L, const Side<T>& R, T (&Fh)[5]) {
  const T sm = L.s > R.s ? L.s : R.s;
#pragma unroll
  for (int q = 0; q < 5; ++q) Fh[q] = fma_(-sm, R.u[q] - L.u[q], L.f[q] + R.f[q]);
}

// One step of every grid.  A block takes tiles of 32 x 8 cells in (x, y) and
// up to 32 planes in z: plane by plane it fills the next plane's tile (cells
// with a one-cell periodic halo in x and y: state, fluxes, wave speeds, each
// computed once) into a double-buffered shared-memory plane, then updates its
// own cells from the four x/y faces of the current plane and the z faces,
// carrying the lower z face of the next plane in registers.
// The scalar step kernel serves FP64 grids (compiler's choice of registers);
// FP32 grids run the packed two-plane kernel k_fv_rusanov_step2 below.

template <class T>
__global__ void __launch_bounds__(kFvThreads) k_fv_rusanov_step(const __grid_constant__ FvArgs a) {
  extern __shared__ __align__(16) unsigned char fv_smem[];
  PlaneTile<T>* tiles = reinterpret_cast<PlaneTile<T>*>(fv_smem);  // [2]
  const Consts<T> k = fv_consts<T>(a.gamma);
  const int tid = threadIdx.x, lx = tid % kBX, ly = tid / kBX;
  const int own = (ly + 1) * kSX + (lx + 1);
  for (int64_t vt = blockIdx.x; vt < a.tiles; vt += gridDim.x) {
    const int gi = find_tile_grid(a, vt);
    const fdbb_fv_grid& g = a.g[gi];
    const int n = g.n;
    const int ntx = ceil_div(n, kBX), nty = ceil_div(n, kBY);
    int64_t loc = vt - a.tile_begin[gi];
    const int tx = (int)(loc % ntx);
    loc /= ntx;
    const int ty = (int)(loc % nty);
    const int tz = (int)(loc / nty);
    const int x0 = tx * kBX, y0 = ty * kBY, z0 = tz * a.zseg;
    const int z1 = z0 + a.zseg < n ? z0 + a.zseg : n;
    T* smax = static_cast<T*>(a.smax) + 3 * g.slot;
    const int ph = g.phase, ph1 = ph == 2 ? 0 : ph + 1, ph2 = ph1 == 2 ? 0 : ph1 + 1;
    const T dx = T(1) / T(n);
    const T dt = T(a.cfl) * dx / smax[ph];
    const T hlam = T(0.5f) * (dt / dx);  // 1/2 of dt/dx: the faces carry twice the flux
    if (tx == 0 && ty == 0 && tz == 0 && tid == 0) {  // the grid's first tile
      smax[ph2] = T(0);  // read by the previous step, filled by the next one
      if (g.dt_log) g.dt_log[g.step] = static_cast<double>(dt);
    }
    const int x = x0 + lx, y = y0 + ly;
    const bool active = x < n && y < n;
    // this thread's slots of a plane tile: cells with a periodic halo; their
    // (x, y) offsets within a plane are the same for every plane of the tile
    int64_t slot_off[kSlotsPerThread];
#pragma unroll
    for (int j = 0; j < kSlotsPerThread; ++j) {
      const int sl = tid + j * kFvThreads;
      const int gx = (x0 + sl % kSX - 1 + n) % n, gy = (y0 + sl / kSX - 1 + n) % n;
      slot_off[j] = (int64_t)gy * n + gx;
    }
    const int64_t plane = (int64_t)n * n;
    auto load_plane = [&](SlotRaw<T>& r, int z) {
      const int64_t zoff = (int64_t)z * plane;
#pragma unroll
      for (int j = 0; j < kSlotsPerThread; ++j) {
        const int sl = tid + j * kFvThreads;
        if (sl < kSlots) {
#pragma unroll
          for (int q = 0; q < 5; ++q) r.u[j][q] = ldg_in<T>(a.dbg, g.U[q], zoff + slot_off[j], plane * n);
        }
      }
    };
    auto fill = [&](PlaneTile<T>& P, const SlotRaw<T>& r) {
#pragma unroll
      for (int j = 0; j < kSlotsPerThread; ++j) {
        const int sl = tid + j * kFvThreads;
        if (sl < kSlots) put_slot<T>(r.u[j], k, P, sl);
      }
    };
    SlotRaw<T> raw;
    load_plane(raw, z0);
    fill(tiles[0], raw);
    load_plane(raw, z0 + 1 == n ? 0 : z0 + 1);  // in flight during the prologue
    // lower z face of the first plane: the own cell of plane z0 - 1 (periodic)
    T zlo[5];
    __syncthreads();
    if (active) {
      PlaneTile<T>& P1 = tiles[1];  // its own slot only, as scratch for the face
      T u[5];
      load_cell<T>(a, g, x, y, z0 == 0 ? n - 1 : z0 - 1, u);
      put_slot<T>(u, k, P1, own);
      face<T>(side<T, 2>(P1, own), side<T, 2>(tiles[0], own), zlo);
    }
    __syncthreads();
    T vmax = T(0);
    for (int z = z0; z < z1; ++z) {
      const PlaneTile<T>& C = tiles[(z - z0) & 1];
      PlaneTile<T>& N = tiles[((z - z0) & 1) ^ 1];
      fill(N, raw);  // plane z + 1
      if (z + 1 < z1) load_plane(raw, z + 2 >= n ? z + 2 - n : z + 2);  // prefetch plane z + 2
      __syncthreads();
      if (active) {
        T lo[5], hi[5], div[5];
        const Cell<T> me = cell_at(C, own);  // the cell's own state, read once
        const T(&uc)[5] = me.u;
        const Side<T> cx = side<T, 0>(me);
        face<T>(side<T, 0>(C, own - 1), cx, lo);
        face<T>(cx, side<T, 0>(C, own + 1), hi);
#pragma unroll
        for (int q = 0; q < 5; ++q) div[q] = T(0) + (hi[q] - lo[q]);
        const Side<T> cy = side<T, 1>(me);
        face<T>(side<T, 1>(C, own - kSX), cy, lo);
        face<T>(cy, side<T, 1>(C, own + kSX), hi);
#pragma unroll
        for (int q = 0; q < 5; ++q) div[q] = div[q] + (hi[q] - lo[q]);
        face<T>(side<T, 2>(me), side<T, 2>(N, own), hi);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          div[q] = div[q] + (hi[q] - zlo[q]);
          zlo[q] = hi[q];
        }
        const int64_t c = ((int64_t)z * n + y) * n + x;
        Pt<T, 3> Nw;
        T un[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          un[q] = fma_(-hlam, div[q], uc[q]);
          st_in<T>(a.dbg, g.Unew[q], c, plane * n, un[q]);
        }
        Nw.rho = un[0];
        Nw.m[0] = un[1];
        Nw.m[1] = un[2];
        Nw.m[2] = un[3];
        Nw.rE = un[4];
        fv_derive(Nw, k);
        const T w = wave_speed_sum(Nw);
        vmax = w > vmax ? w : vmax;
      }
      __syncthreads();  // the next iteration refills the current plane
    }
    vmax = warp_max(vmax);
    if ((tid & 31) == 0 && vmax > T(0)) atomic_max_pos(smax + ph1, vmax);
  }
}

// ---------------------------------------------------------------------------
// FP32 grids: two planes per thread in packed FP32x2 arithmetic.
//
// A thread updates the same (x, y) cell of planes z and z + 1: lane x of each
// packed value belongs to plane z, lane y to plane z + 1 (z - z0 even; the
// segments start at multiples of the segment length, which is even, so a plane has the same
// lane in every tile).  Every operation of the faces, the update and the
// derived state then takes one packed instruction (FFMA2 / FADD2 / FMUL2 of
// sm_100 and later) for two cells.  Each lane rounds like the scalar FP32
// operation, and a face computed by two threads or two tiles goes through
// the same packed sequence on the same inputs, so its two copies agree bit for
// bit and the update conserves mass, momentum and energy to rounding.
// ---------------------------------------------------------------------------
struct f2 {
  float2 v;
};
__device__ __forceinline__ f2 pk(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ f2 splat(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return {__fmul2_rn(a.v, b.v)}; }
// a - b as (-1) b + a: the product is exact, so one rounding as in a subtraction
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return {__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)}; }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ f2 abs2(f2 a) { return pk(fabsf(a.v.x), fabsf(a.v.y)); }
__device__ __forceinline__ f2 max2(f2 a, f2 b) {
  return pk(a.v.x > b.v.x ? a.v.x : b.v.x, a.v.y > b.v.y ? a.v.y : b.v.y);
}

// Plane-pair tile: for each of the kSlots cells of a (32+2) x (8+2) tile,
// U, p, 1/rho and c of planes z and z + 1, as four float4 per slot --
// (rho, m_x), (m_y, m_z), (rhoE, p), (1/rho, c), each value as its
// (plane z, plane z + 1) pair: half the shared-memory instructions of one
// float2 per value.  The kernel keeps a ring of three (3 x 21.8 KB).
struct PairTile {
  float4 v[kSlotVals / 2][kSlots];
};
constexpr int kPairRing = 3;
struct Cell2 {
  f2 u[5], p, r, c;
};
struct Consts2 {
  f2 a1, g, half;
};

// U, p, 1/rho and c of a pair of cells (the scalar FP32 derivation, packed).
__device__ __forceinline__ Cell2 derive2(const f2 (&u)[5], const Consts2& k) {
  Cell2 e;
#pragma unroll
  for (int q = 0; q < 5; ++q) e.u[q] = u[q];
  e.r = pk(fv_rcp(u[0].v.x), fv_rcp(u[0].v.y));
  // p = (gamma - 1) (rhoE - |m|^2 / (2 rho))
  const f2 m2 = fma2(u[3], u[3], fma2(u[2], u[2], u[1] * u[1]));
  e.p = k.a1 * (u[4] - k.half * (m2 * e.r));
  const f2 c2 = k.g * e.p * e.r;
  e.c = pk(fv_sqrt(c2.v.x), fv_sqrt(c2.v.y));
  return e;
}
__device__ __forceinline__ float4 q4(f2 a, f2 b) { return make_float4(a.v.x, a.v.y, b.v.x, b.v.y); }
__device__ __forceinline__ void put_pair(const Cell2& e, PairTile& P, int slot) {
  P.v[0][slot] = q4(e.u[0], e.u[1]);
  P.v[1][slot] = q4(e.u[2], e.u[3]);
  P.v[2][slot] = q4(e.u[4], e.p);
  P.v[3][slot] = q4(e.r, e.c);
}
__device__ __forceinline__ Cell2 pair_at(const PairTile& P, int slot) {
  const float4 a = P.v[0][slot], b = P.v[1][slot], c = P.v[2][slot], d = P.v[3][slot];
  Cell2 e;
  e.u[0] = pk(a.x, a.y);
  e.u[1] = pk(a.z, a.w);
  e.u[2] = pk(b.x, b.y);
  e.u[3] = pk(b.z, b.w);
  e.u[4] = pk(c.x, c.y);
  e.p = pk(c.z, c.w);
  e.r = pk(d.x, d.y);
  e.c = pk(d.z, d.w);
  return e;
}

// Face side in direction d: U, F_d(U) and |v_d| + c (as side<T, d>).
struct Side2 {
  f2 u[5], f[5], s;
};
template <int d> __device__ __forceinline__ Side2 side2(const Cell2& e) {
  Side2 x;
  const f2 md = e.u[1 + d];
#pragma unroll
  for (int q = 0; q < 5; ++q) x.u[q] = e.u[q];
  x.f[0] = md;
  // m_i v_d for every momentum component, the pressure added to the normal one
  const f2 vd = md * e.r;
#pragma unroll
  for (int i = 0; i < 3; ++i) x.f[1 + i] = i == d ? fma2(md, vd, e.p) : e.u[1 + i] * vd;
  x.f[4] = vd * (e.u[4] + e.p);
  x.s = abs2(vd) + e.c;
  return x;
}
// Twice the Rusanov flux, (F(U_L) + F(U_R)) + s (U_L - U_R) (as face<T>).
__device__ __forceinline__ void face2(const Side2& L, const Side2& R, f2 (&Fh)[5]) {
  const f2 sm = max2(L.s, R.s);
#pragma unroll
  for (int q = 0; q < 5; ++q) Fh[q] = fma2(sm, L.u[q] - R.u[q], L.f[q] + R.f[q]);
}

// Conservative values of this thread's slots of a plane pair.
struct PairRaw {
  f2 u[kSlotsPerThread][5];
};

__global__ void __launch_bounds__(kFvThreads, 2) k_fv_rusanov_step2(const __grid_constant__ FvArgs a) {
  extern __shared__ __align__(16) unsigned char fv_smem[];
  PairTile* tiles = reinterpret_cast<PairTile*>(fv_smem);  // ring of kPairRing
  const Consts<float> k1 = fv_consts<float>(a.gamma);
  const Consts2 k = {splat(k1.a1), splat(k1.g), splat(0.5f)};
  const int tid = threadIdx.x, lx = tid % kBX, ly = tid / kBX;
  const int own = (ly + 1) * kSX + (lx + 1);
  for (int64_t vt = blockIdx.x; vt < a.tiles; vt += gridDim.x) {
    const int gi = find_tile_grid(a, vt);
    const fdbb_fv_grid& g = a.g[gi];
    const int n = g.n;
    const int ntx = ceil_div(n, kBX), nty = ceil_div(n, kBY);
    int64_t loc = vt - a.tile_begin[gi];
    const int tx = (int)(loc % ntx);
    loc /= ntx;
    const int ty = (int)(loc % nty);
    const int tz = (int)(loc / nty);
    const int x0 = tx * kBX, y0 = ty * kBY, z0 = tz * a.zseg;
    const int z1 = z0 + a.zseg < n ? z0 + a.zseg : n;
    float* smax = static_cast<float*>(a.smax) + 3 * g.slot;
    const int ph = g.phase, ph1 = ph == 2 ? 0 : ph + 1, ph2 = ph1 == 2 ? 0 : ph1 + 1;
    const float dx = 1.0f / float(n);
    const float dt = float(a.cfl) * dx / smax[ph];
    const f2 mhlam = splat(-(0.5f * (dt / dx)));  // -1/2 dt/dx: the faces carry twice the flux
    if (tx == 0 && ty == 0 && tz == 0 && tid == 0) {  // the grid's first tile
      smax[ph2] = 0.0f;  // read by the previous step, filled by the next one
      if (g.dt_log) g.dt_log[g.step] = static_cast<double>(dt);
    }
    const int x = x0 + lx, y = y0 + ly;
    const bool active = x < n && y < n;
    int64_t slot_off[kSlotsPerThread];
#pragma unroll
    for (int j = 0; j < kSlotsPerThread; ++j) {
      const int sl = tid + j * kFvThreads;
      const int gx = (x0 + sl % kSX - 1 + n) % n, gy = (y0 + sl / kSX - 1 + n) % n;
      slot_off[j] = (int64_t)gy * n + gx;
    }
    const int64_t plane = (int64_t)n * n;
    // z mod n for 0 <= z < n + 6: one compare and subtract (a modulo by the
    // run-time n is an integer-division sequence; only grids of n <= 5 need it)
    auto wrap = [n](int z) {
      const int w = z - n;
      return z < n ? z : (w < n ? w : w % n);
    };
    // planes za (lane x) and zb (lane y) of this thread's slots
    auto load_pair = [&](PairRaw& r, int za, int zb) {
      const int64_t oa = (int64_t)za * plane, ob = (int64_t)zb * plane;
#pragma unroll
      for (int j = 0; j < kSlotsPerThread; ++j) {
        const int sl = tid + j * kFvThreads;
        if (sl < kSlots) {
#pragma unroll
          for (int q = 0; q < 5; ++q)
            r.u[j][q] = pk(ldg_in<float>(a.dbg, g.U[q], oa + slot_off[j], plane * n),
                           ldg_in<float>(a.dbg, g.U[q], ob + slot_off[j], plane * n));
        }
      }
    };
    auto fill = [&](PairTile& P, const PairRaw& r) {
#pragma unroll
      for (int j = 0; j < kSlotsPerThread; ++j) {
        const int sl = tid + j * kFvThreads;
        if (sl < kSlots) put_pair(derive2(r.u[j], k), P, sl);
      }
    };
    PairRaw raw;
    load_pair(raw, z0, wrap(z0 + 1));
    fill(tiles[0], raw);
    load_pair(raw, wrap(z0 + 2), wrap(z0 + 3));  // in flight during the prologue
    __syncthreads();
    // lower z face of plane z0, from the cells of planes z0 - 1 and z0 (lane x;
    // the same packed sequence as the upper faces of the tile below)
    f2 carry[5];
    if (active) {
      const int64_t cm = (int64_t)(z0 == 0 ? n - 1 : z0 - 1) * plane + (int64_t)y * n + x;
      f2 um[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) um[q] = splat(ldg_in<float>(a.dbg, g.U[q], cm, plane * n));
      const Cell2 lower = derive2(um, k);
      Cell2 cur = pair_at(tiles[0], own);
#pragma unroll
      for (int q = 0; q < 5; ++q) cur.u[q] = splat(cur.u[q].v.x);
      cur.p = splat(cur.p.v.x);
      cur.r = splat(cur.r.v.x);
      cur.c = splat(cur.c.v.x);
      face2(side2<2>(lower), side2<2>(cur), carry);
    }
    float vmax = 0.0f;
    // Pair tiles in a ring of three: iteration i reads tiles i and i + 1 and
    // fills tile i + 1, whose previous contents (tile i - 2) every thread
    // finished reading before the barrier of iteration i - 1; one barrier per
    // plane pair.
    for (int z = z0, b = 0; z < z1; z += 2, b = b == kPairRing - 1 ? 0 : b + 1) {
      const PairTile& C = tiles[b];
      PairTile& N = tiles[b == kPairRing - 1 ? 0 : b + 1];
      fill(N, raw);  // planes z + 2, z + 3
      if (z + 2 < z1) load_pair(raw, wrap(z + 4), wrap(z + 5));  // prefetch planes z + 4, z + 5
      __syncthreads();
      if (active) {
        const bool two = z + 1 < z1;  // lane y is a cell of this segment
        f2 lo[5], hi[5], div[5];
        const Cell2 me = pair_at(C, own);
        const Side2 cx = side2<0>(me);
        face2(side2<0>(pair_at(C, own - 1)), cx, lo);
        face2(cx, side2<0>(pair_at(C, own + 1)), hi);
#pragma unroll
        for (int q = 0; q < 5; ++q) div[q] = hi[q] - lo[q];
        const Side2 cy = side2<1>(me);
        face2(side2<1>(pair_at(C, own - kSX)), cy, lo);
        face2(cy, side2<1>(pair_at(C, own + kSX)), hi);
#pragma unroll
        for (int q = 0; q < 5; ++q) div[q] = div[q] + (hi[q] - lo[q]);
        // z faces: upper faces of planes z and z + 1 from the cells of planes
        // (z + 1, z + 2); the lower faces are (carry, upper face of plane z)
        const Cell2 nx = pair_at(N, own);
        Cell2 up;
#pragma unroll
        for (int q = 0; q < 5; ++q) up.u[q] = pk(me.u[q].v.y, nx.u[q].v.x);
        up.p = pk(me.p.v.y, nx.p.v.x);
        up.r = pk(me.r.v.y, nx.r.v.x);
        up.c = pk(me.c.v.y, nx.c.v.x);
        face2(side2<2>(me), side2<2>(up), hi);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          div[q] = div[q] + (hi[q] - pk(carry[q].v.x, hi[q].v.x));
          carry[q] = splat(hi[q].v.y);
        }
        const int64_t c = ((int64_t)z * n + y) * n + x;
        f2 un[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          un[q] = fma2(mhlam, div[q], me.u[q]);
          st_in<float>(a.dbg, g.Unew[q], c, plane * n, un[q].v.x);
          if (two) st_in<float>(a.dbg, g.Unew[q], c + plane, plane * n, un[q].v.y);
        }
        const Cell2 nw = derive2(un, k);
        // sum over d of |v_d| + c as (|m_x| + |m_y| + |m_z|) / rho + 3 c
        const f2 vs = fma2(abs2(un[1]) + abs2(un[2]) + abs2(un[3]), nw.r, splat(3.0f) * nw.c);
        vmax = vs.v.x > vmax ? vs.v.x : vmax;
        if (two) vmax = vs.v.y > vmax ? vs.v.y : vmax;
      }
    }
    __syncthreads();  // the next tile's prologue refills the ring
    vmax = warp_max(vmax);
    if ((tid & 31) == 0 && vmax > 0.0f) atomic_max_pos(smax + ph1, vmax);
  }
}

constexpr size_t fv_step_smem(size_t es) { return 2 * (size_t)kSlotVals * kSlots * es; }

// Step kernel and its dynamic shared memory for storage T: FP32 grids take
// the packed two-plane kernel, FP64 grids the scalar one.
template <class T> auto step_kernel() {
  if constexpr (std::is_same<T, float>::value)
    return k_fv_rusanov_step2;
  else
    return k_fv_rusanov_step<T>;
}
template <class T> constexpr size_t step_smem() {
  return std::is_same<T, float>::value ? kPairRing * sizeof(PairTile) : fv_step_smem(sizeof(T));
}

// Resident blocks per SM of the step (step = true, after its opt-in to more
// than 48 KB of dynamic shared memory) or wave-speed kernel on the current
// device.  Function attributes belong to each device's context, so the opt-in
// and the occupancy are taken, and cached, per device.
template <class T> int fv_blocks_per_sm(bool step) {
  static std::atomic<int> cache[2][kMaxDevices];
  const int slot = current_device_slot();
  if (slot >= 0) {
    const int v = cache[step][slot].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int b = 0;
  cudaError_t e = cudaSuccess;
  if (step) {
    e = cudaFuncSetAttribute(step_kernel<T>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step_smem<T>());
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, step_kernel<T>(), kFvThreads, step_smem<T>());
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fv_max_speed<T>, kFvThreads, 0);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    b = 1;
  }
  if (b <= 0) b = 1;
  if (slot >= 0 && e == cudaSuccess) cache[step][slot].store(b, std::memory_order_relaxed);
  return b;
}

// Planes per column segment of the step kernel: the longest of 64, 32 and 16
// that still gives every resident block at least three tiles.  Longer
// segments spend less on each tile's prologue (8 grids of 128^3 on one
// GB300: 16 planes 6.13e10, 32: 6.54e10, 64: 6.93e10, 128: 5.99e10
// cell-steps/s); shorter ones keep every SM busy when few cells are stepped.
// The results do not depend on it: every face is the same computation in any
// segmentation.  Sets a.zseg and the tile table.
template <class T> void fv_plan(FvArgs& a) {
  const int64_t cap = (int64_t)device_sm_count() * fv_blocks_per_sm<T>(true);
  for (int z : {64, 32, 16}) {
    a.zseg = z;
    fv_tiles(a);
    if (a.tiles >= 3 * cap) return;
  }
}

template <class T> cudaError_t fv_launch(const FvArgs& a, bool step, cudaStream_t s) {
  const int64_t work = step ? a.tiles : a.vcells / kFvThreads;
  const int64_t cap = (int64_t)device_sm_count() * fv_blocks_per_sm<T>(step);
  const int grid = (int)(work < cap ? work : cap);
  if (grid <= 0) return cudaSuccess;
  if (step)
    step_kernel<T>()<<<grid, kFvThreads, step_smem<T>(), s>>>(a);
  else
    k_fv_max_speed<T><<<grid, kFvThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Smooth periodic initial state (the serving workload's requests)
// ---------------------------------------------------------------------------

// The two sums of three sinusoids, g_r = sum_m a sin(2 pi k.x + phi).
struct SmoothArgs {
  void* U[5];
  int n;
  double w[2][3][5];  // [plane][sinusoid]: k_x, k_y, k_z, phase, amplitude
  double amp, ia1;
};

__device__ __forceinline__ float sin_(float x) { return sinf(x); }
__device__ __forceinline__ double sin_(double x) { return sin(x); }

template <class T> __device__ __forceinline__ void smooth_g(const SmoothArgs& a, int64_t c, T (&g)[2]) {
  const int n = a.n;
  const int i = (int)(c % n), j = (int)((c / n) % n), kz = (int)(c / ((int64_t)n * n));
  const T x = (T(i) + T(0.5f)) / T(n), y = (T(j) + T(0.5f)) / T(n), z = (T(kz) + T(0.5f)) / T(n);
  const T tp = T(6.283185307179586);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    T acc = T(0);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const double* w = a.w[r][m];
      const T arg = tp * (T(w[0]) * x + T(w[1]) * y + T(w[2]) * z) + T(w[3]);
      acc = acc + T(w[4]) * sin_(arg);
    }
    g[r] = acc;
  }
}

template <class T>
__global__ void __launch_bounds__(kFvThreads) k_fv_smooth_max(const __grid_constant__ SmoothArgs a, T* gmax) {
  const int64_t cells = (int64_t)a.n * a.n * a.n;
  T m0 = T(0), m1 = T(0);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (int64_t)gridDim.x * blockDim.x) {
    T g[2];
    smooth_g(a, c, g);
    m0 = abs_(g[0]) > m0 ? abs_(g[0]) : m0;
    m1 = abs_(g[1]) > m1 ? abs_(g[1]) : m1;
  }
  m0 = warp_max(m0);
  m1 = warp_max(m1);
  if ((threadIdx.x & 31) == 0) {
    if (m0 > T(0)) atomic_max_pos(gmax + 0, m0);
    if (m1 > T(0)) atomic_max_pos(gmax + 1, m1);
  }
}

template <class T>
__global__ void __launch_bounds__(kFvThreads) k_fv_smooth_write(const __grid_constant__ SmoothArgs a, const T* gmax) {
  const int64_t cells = (int64_t)a.n * a.n * a.n;
  const T s0 = T(a.amp) / gmax[0], s1 = T(a.amp) / gmax[1], ia1 = T(a.ia1);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (int64_t)gridDim.x * blockDim.x) {
    T g[2];
    smooth_g(a, c, g);
    static_cast<T*>(a.U[0])[c] = fma_(s0, g[0], T(1));
    static_cast<T*>(a.U[1])[c] = T(0);
    static_cast<T*>(a.U[2])[c] = T(0);
    static_cast<T*>(a.U[3])[c] = T(0);
    static_cast<T*>(a.U[4])[c] = fma_(s1, g[1], T(1)) * ia1;
  }
}

template <class T> cudaError_t smooth_launch(const SmoothArgs& a, void* scratch, cudaStream_t s) {
  const int64_t cells = (int64_t)a.n * a.n * a.n;
  const int64_t need = (cells + kFvThreads - 1) / kFvThreads;
  const int64_t cap = (int64_t)device_sm_count() * 8;
  const int grid = (int)(need < cap ? need : cap);
  cudaError_t e = cudaMemsetAsync(scratch, 0, 2 * sizeof(T), s);
  if (e != cudaSuccess) return e;
  k_fv_smooth_max<T><<<grid, kFvThreads, 0, s>>>(a, static_cast<T*>(scratch));
  k_fv_smooth_write<T><<<grid, kFvThreads, 0, s>>>(a, static_cast<const T*>(scratch));
  return cudaGetLastError();
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// Host-side checks of a grid table: sorted, tile-aligned, non-overlapping
// ranges inside [0, vcells), non-NULL aligned planes, U and Unew distinct.
fdbb_status fv_check(int ngrids, const fdbb_fv_grid* grids, int64_t vcells, fdbb_dtype t, const void* smax,
                     bool step, int64_t* slots_out) {
  if (ngrids < 0 || ngrids > FDBB_FV_MAX_GRIDS || vcells < 0 || vcells % FDBB_FV_TILE) return FDBB_ERR_ARG;
  if (t != FDBB_F32 && t != FDBB_F64) return FDBB_ERR_DTYPE;
  if (ngrids > 0 && (grids == nullptr || smax == nullptr)) return FDBB_ERR_NULLPTR;
  if (smax && !aligned(smax, t == FDBB_F64 ? 8 : 4)) return FDBB_ERR_ALIGN;
  const size_t es = t == FDBB_F64 ? 8 : 4;
  int64_t end = 0, slots = 0;
  for (int i = 0; i < ngrids; ++i) {
    const fdbb_fv_grid& g = grids[i];
    if (g.n < 1 || g.n > 4096 || g.slot < 0 || g.phase < 0 || g.phase > 2 || g.step < 0) return FDBB_ERR_ARG;
    const int64_t cells = (int64_t)g.n * g.n * g.n;
    const int64_t padded = (cells + FDBB_FV_TILE - 1) / FDBB_FV_TILE * FDBB_FV_TILE;
    if (g.cell_begin < end || g.cell_begin % FDBB_FV_TILE || g.cell_begin + padded > vcells) return FDBB_ERR_ARG;
    end = g.cell_begin + padded;
    for (int q = 0; q < 5; ++q) {
      if (g.U[q] == nullptr || (step && g.Unew[q] == nullptr)) return FDBB_ERR_NULLPTR;
      if (!aligned(g.U[q], es) || (step && !aligned(g.Unew[q], es))) return FDBB_ERR_ALIGN;
      if (step)
        for (int r = 0; r < 5; ++r)
          if (g.Unew[q] == g.U[r]) return FDBB_ERR_ARG;
    }
    if (g.dt_log && !aligned(g.dt_log, 8)) return FDBB_ERR_ALIGN;
    if (g.slot + 1 > slots) slots = g.slot + 1;
  }
  if (slots_out) *slots_out = slots;
  return FDBB_OK;
}

fdbb_status fv_run(int ngrids, const fdbb_fv_grid* grids, int64_t vcells, double gamma, double cfl, fdbb_dtype t,
                   void* smax, bool step, fdbb_stream_t stream) {
  if (!(gamma > 1.0) || !std::isfinite(gamma)) return FDBB_ERR_ARG;
  if (step && !(cfl > 0.0 && std::isfinite(cfl))) return FDBB_ERR_ARG;
  const fdbb_status st = fv_check(ngrids, grids, vcells, t, smax, step, nullptr);
  if (st != FDBB_OK) return st;
  if (ngrids == 0 || vcells == 0) return FDBB_OK;
  FvArgs a;
  a.ngrids = ngrids;
  a.vcells = vcells;
  a.gamma = gamma;
  a.cfl = cfl;
  a.smax = smax;
  a.dbg = debug_counters();
  for (int i = 0; i < ngrids; ++i) a.g[i] = grids[i];
  if (t == FDBB_F64)
    fv_plan<double>(a);
  else
    fv_plan<float>(a);
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const cudaError_t e = t == FDBB_F64 ? fv_launch<double>(a, step, s) : fv_launch<float>(a, step, s);
  return e == cudaSuccess ? FDBB_OK : FDBB_ERR_CUDA;
}

// Scratch of fdbb_fv_rusanov_step_noalloc: three wave-speed slots for each of
// at most FDBB_FV_MAX_GRIDS grids (6 KiB).  It lives in every device that loads
// the library, for as long as the library stays loaded, and is shared by every
// call of that entry point on that device.
static __device__ __align__(256) double g_fv_noalloc_smax[3 * FDBB_FV_MAX_GRIDS];

// Device address of g_fv_noalloc_smax on the current device.  In host code the
// symbol's name is a host-side stand-in, not a device address, so the address
// is looked up with cudaGetSymbolAddress, with the device current, the first
// time the entry point runs on that device, and cached by device number for
// the rest of the process (a device reset would invalidate it; the header
// says so).
fdbb_status noalloc_scratch(void** out) {
  static std::mutex mu;
  static std::unordered_map<int, void*> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FDBB_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(mu);
  const auto it = cache.find(dev);
  if (it != cache.end()) {
    *out = it->second;
    return FDBB_OK;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_fv_noalloc_smax) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return FDBB_ERR_CUDA;
  }
  cache.emplace(dev, p);
  *out = p;
  return FDBB_OK;
}

fdbb_status fv_step_noalloc(int ngrids, const fdbb_fv_grid* grids, int64_t vcells, double gamma, double cfl,
                            fdbb_dtype t, fdbb_stream_t stream) {
  if (ngrids > FDBB_FV_MAX_GRIDS) return FDBB_ERR_ARG;  // beyond the static scratch
  if (ngrids < 0 || !(gamma > 1.0) || !std::isfinite(gamma) || !(cfl > 0.0 && std::isfinite(cfl)))
    return FDBB_ERR_ARG;
  if (ngrids > 0 && grids == nullptr) return FDBB_ERR_NULLPTR;
  FvArgs a;
  a.ngrids = ngrids;
  a.vcells = vcells;
  a.gamma = gamma;
  a.cfl = cfl;
  for (int i = 0; i < ngrids; ++i) {
    a.g[i] = grids[i];
    a.g[i].slot = i;   // slot and phase of the caller's table are not used:
    a.g[i].phase = 0;  // every call recomputes the wave speed of U
  }
  // Arguments first, before any CUDA call; the scratch pointer is not known
  // yet, so the check sees a stand-in with the array's alignment.
  alignas(256) static const double kStandIn = 0.0;
  const fdbb_status st = fv_check(ngrids, a.g, vcells, t, &kStandIn, true, nullptr);
  if (st != FDBB_OK) return st;
  if (ngrids == 0 || vcells == 0) return FDBB_OK;
  void* scratch = nullptr;
  const fdbb_status sst = noalloc_scratch(&scratch);
  if (sst != FDBB_OK) return sst;
  a.smax = scratch;
  a.dbg = debug_counters();
  if (t == FDBB_F64)
    fv_plan<double>(a);
  else
    fv_plan<float>(a);
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the slots keep the previous call's contents: clear them first
  if (cudaMemsetAsync(scratch, 0, sizeof(double) * 3 * (size_t)ngrids, s) != cudaSuccess) {
    cudaGetLastError();
    return FDBB_ERR_CUDA;
  }
  cudaError_t e = t == FDBB_F64 ? fv_launch<double>(a, false, s) : fv_launch<float>(a, false, s);
  if (e == cudaSuccess) e = t == FDBB_F64 ? fv_launch<double>(a, true, s) : fv_launch<float>(a, true, s);
  return e == cudaSuccess ? FDBB_OK : FDBB_ERR_CUDA;
}

}  // namespace
}  // namespace fdbb

extern "C" {

fdbb_status fdbb_fv_init_smooth(const fdbb_fv_grid* grid, double gamma, double amplitude, const double* wave,
                                fdbb_dtype t, void* scratch, fdbb_stream_t stream) {
  using namespace fdbb;
  if (grid == nullptr || wave == nullptr || scratch == nullptr) return FDBB_ERR_NULLPTR;
  if (t != FDBB_F32 && t != FDBB_F64) return FDBB_ERR_DTYPE;
  if (grid->n < 1 || grid->n > 4096 || !(gamma > 1.0) || !std::isfinite(gamma) || !std::isfinite(amplitude))
    return FDBB_ERR_ARG;
  const uintptr_t al = t == FDBB_F64 ? 8 : 4;
  if (!aligned(scratch, al)) return FDBB_ERR_ALIGN;
  SmoothArgs a = {};
  for (int q = 0; q < 5; ++q) {
    if (grid->U[q] == nullptr) return FDBB_ERR_NULLPTR;
    if (!aligned(grid->U[q], 16)) return FDBB_ERR_ALIGN;
    a.U[q] = grid->U[q];
  }
  for (int r = 0; r < 2; ++r)
    for (int m = 0; m < 3; ++m)
      for (int f = 0; f < 5; ++f) {
        const double v = wave[15 * r + 5 * m + f];
        if (!std::isfinite(v)) return FDBB_ERR_ARG;
        a.w[r][m][f] = v;
      }
  a.n = grid->n;
  a.amp = amplitude;
  a.ia1 = 1.0 / (gamma - 1.0);
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const cudaError_t e = t == FDBB_F64 ? smooth_launch<double>(a, scratch, s) : smooth_launch<float>(a, scratch, s);
  return e == cudaSuccess ? FDBB_OK : FDBB_ERR_CUDA;
}

fdbb_status fdbb_fv_rusanov_step_noalloc(int ngrids, const fdbb_fv_grid* grids, int64_t vcells, double gamma,
                                         double cfl, fdbb_dtype t, fdbb_stream_t stream) {
  return fdbb::fv_step_noalloc(ngrids, grids, vcells, gamma, cfl, t, stream);
}

fdbb_status fdbb_fv_max_speed(int ngrids, const fdbb_fv_grid* grids, int64_t vcells, double gamma, fdbb_dtype t,
                              void* smax, fdbb_stream_t stream) {
  return fdbb::fv_run(ngrids, grids, vcells, gamma, 1.0, t, smax, false, stream);
}

fdbb_status fdbb_fv_rusanov_step(int ngrids, const fdbb_fv_grid* grids, int64_t vcells, double gamma, double cfl,
                                 fdbb_dtype t, void* smax, fdbb_stream_t stream) {
  return fdbb::fv_run(ngrids, grids, vcells, gamma, cfl, t, smax, true, stream);
}

}  // extern "C"
