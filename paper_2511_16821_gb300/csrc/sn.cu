// sn.cu -- collided S_N-DG stage (Sec. 2.2 step 2, Eq. (floor N_s+1)) on sm_103a.
//
// Backward Euler from zero data with vacuum boundaries:
//   (sigma_t + 1/(c dt)) Psi_c + Omega.grad Psi_c = (sigma_s / 4 pi)(phi_c + phi_{N_s}),
// where the fixed part comes from the hand-off moments m_i = sigma_s sum w int P_i ds (space-time
// integrals, so the source integral against P_i is m_i / (4 pi dt)). Bilinear DG per cell,
// psi = a0 + a1 xi + a2 eta + a3 xi eta, upwind traces, level-symmetric quadrature; source
// iteration on phi_c.
//
// Sweep: one CTA per ordinate; its warps walk 32-row strips as wavefronts (lane = row, one
// anti-diagonal per step); the trace entering a row from below comes from the neighbouring lane by
// shuffle (from the strip below through a shared-memory ring), the trace from the left stays in
// registers, so a step needs no block barrier. The sources live on a mesh padded with zero halo
// columns and an extra row, the solutions on the plain mesh behind predicated stores (or, for
// solves too large for L2, both in the sweep's own wavefront order), so a step needs no bound
// test. Strips are pipelined across the warps, so the critical path is about
// (nx + 31) + (32 + PF - 1)(ceil(ny/32) - 1) cell solves per sweep. Coordinates are mirrored per
// quadrant so that every sweep runs towards +x,+y; in mirrored coordinates the 4x4 cell system is
// the same for every quadrant and is diagonally dominant, so it is solved by elimination without
// pivoting. The per-ordinate results are summed over ordinates in a fixed order (deterministic).
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>
#include <utility>

#include "hyb_device.cuh"
#include "pdl.cuh"

namespace hyb {

// Each sweep and reduction of the source iteration of a problem stepped alone (hyb_problem::pdl) is
// launched as a programmatic dependent of its predecessor (pdl.cuh): it waits for the predecessor
// before reading, and lets its successor be scheduled as soon as it starts.

// Padded mesh of the sweep's sources: every row carries kHalo columns on both sides, and one extra
// row follows the last; halo and extra row are zero. A lane before its row's first column, past its
// last, or on a row beyond the mesh then loads zero data without a bound test, and a cell solve with
// zero data and zero inflow returns zero traces, so the inflow of column 0 is zero without a reset.
// kHalo covers the columns a lane reads: loads run PF steps ahead of the step, the last block of
// steps overruns the wavefront by up to PF - 1, and lane l trails lane 0 by l. The solutions psi
// stay on the plain mesh: their store is predicated on the lane holding a mesh cell.
//
// PF: the cell data prefetch depth of the sweep, in wavefront steps (a ring of register sets,
// unrolled so that no value moves between registers while its load is in flight), which is also the
// length of the block of steps between two ring waits
template <typename T> struct SweepDepth { static constexpr int value = sizeof(T) == 4 ? 8 : 4; };

template <typename T> struct SweepPad {
    static constexpr int kHalo = 32 + 2 * SweepDepth<T>::value;
    static __host__ __device__ int nxp(int nx) { return nx + 2 * kHalo; }
    static __host__ __device__ size_t plane(int nx, int ny) { return (size_t)(ny + 1) * nxp(nx); }
    static __host__ __device__ size_t at(int nx, int ix, int iy) { return (size_t)iy * nxp(nx) + kHalo + ix; }
};

// Mirror signs of quadrant Q (ordinates m = Q nq + q): the sweep of every quadrant runs towards
// +x, +y in coordinates mirrored by (sx, sy).
__host__ __device__ __forceinline__ int quad_sx(int Q) { return (Q == 0 || Q == 3) ? 1 : -1; }
__host__ __device__ __forceinline__ int quad_sy(int Q) { return Q <= 1 ? 1 : -1; }

// The other memory layout of the sweep, for problems whose solve does not stay in L2: the wavefront
// order of each direction. Entry (s, t, l) -- strip s, step t, lane l -- holds the cell of mirrored
// row 32 s + l and mirrored column t - l, so the 32 lanes of a step read or write 32 consecutive
// entries (one coalesced access to DRAM) and a lane's next step is 32 entries on; the scatter
// between mesh order and this order is done by the fully parallel kernels that write the sources
// and read the solutions. Entries that hold no cell are zero in the source arrays and take the junk
// stores of psi, so a step tests no bound (zero data and zero inflow give zero traces, as on the
// padded mesh). nt covers the last block of steps and the loads PF steps ahead of it. On the padded
// mesh a lane walks its own row, so the lines of consecutive steps are reused from L1; in wavefront
// order every step takes new lines, which costs more than the coalescing saves while the data sit in
// L2 (measured on 112^2 cells, S8: sweep 37 -> 43 us) and saves a fifth of the solve once they do
// not (1024^2 cells: 1.44 -> 1.14 ms per source iteration).
template <typename T> struct Wave {
    int nx, ny, nstrip, nt;
    __host__ __device__ static Wave make(int nx, int ny) {
        constexpr int PF = SweepDepth<T>::value;
        Wave w;
        w.nx = nx; w.ny = ny;
        w.nstrip = (ny + 31) / 32;
        w.nt = (nx + 31 + PF - 1) / PF * PF + PF;
        return w;
    }
    __host__ __device__ size_t size() const { return (size_t)nstrip * nt * 32; }
    // entry of mesh cell (ix, iy) in the direction mirrored by (sx, sy)
    __host__ __device__ size_t at(int ix, int iy, int sx, int sy) const {
        const int ly = sy > 0 ? iy : ny - 1 - iy, c = sx > 0 ? ix : nx - 1 - ix;
        const int l = ly & 31;
        return ((size_t)(ly >> 5) * nt + c + l) * 32 + l;
    }
};

// the wavefront layout is taken when the per-ordinate solutions of the plain mesh exceed this
constexpr size_t kWaveMinPsiBytes = size_t(48) << 20;

bool sn_wave_layout(int nx, int ny, int nord, bool fp64, int layout) {
    if (layout != 0) return layout == 2;
    return (size_t)nord * nx * ny * 4 * (fp64 ? 8 : 4) > kWaveMinPsiBytes;
}

template <typename T>
struct SweepArgs {
    int nx, ny, nq, nord, W, re;   // re: ring entries per slot
    T dx, dy;
    const T* src;            // the four source integrals S_i (un-mirrored): padded mesh, or per direction in
    const T* sgA;            //   wavefront order; (sigma_t + 1/(c dt)) A, the same way
    Wave<T> wv;              // the wavefront layout (used by the wavefront sweep)
    const T* k8;             // cell-solve table (or null): per class q and padded cell k1..k4, Ai, Bi, Di, i0
    const T* i3;             //   and i3
    const T* qox; const T* qoy;    // ordinates by quadrant: m = quad * nq + q
    size_t plane;            // cells per padded plane (rows of the table)
    T* psi;                  // per ordinate, psi (4 Legendre coefficients, mirrored): plain mesh or wavefront
    int* status;             // device status word (bounded waits)
    const int* conv;         // converged flag: set -> the sweep returns at once
    int poll_limit;          // polls of a strip-pipeline wait before it gives up (status kStSegments)
};

// source integrals against P_i: sigma_s A n_i phi_i / (4 pi) + m_i / (4 pi dt)
template <typename T>
__device__ __forceinline__ void source4(T ss, T area, const T* po, const double* mm, T inv_4pi_dt, T* S) {
    const T cs = ss * area * T(0.07957747154594767);   // sigma_s A / (4 pi)
    S[0] = cs * po[0] + (T)mm[0] * inv_4pi_dt;
    S[1] = cs * po[1] * T(1.0 / 3.0) + (T)mm[1] * inv_4pi_dt;
    S[2] = cs * po[2] * T(1.0 / 3.0) + (T)mm[2] * inv_4pi_dt;
    S[3] = cs * po[3] * T(1.0 / 9.0) + (T)mm[3] * inv_4pi_dt;
}

// the sweep entries of cell (ix, iy): one on the padded mesh, one per direction in wavefront order
template <typename T>
__device__ __forceinline__ int sweep_entries(bool wave, const Wave<T>& wv, int nx, int ix, int iy, size_t* e) {
    if (!wave) { e[0] = SweepPad<T>::at(nx, ix, iy); return 1; }
    const size_t wsz = wv.size();
#pragma unroll
    for (int Q = 0; Q < 4; ++Q) e[Q] = (size_t)Q * wsz + wv.at(ix, iy, quad_sx(Q), quad_sy(Q));
    return 4;
}

// The first iteration's sources. The solve's starting iterate is formed here too: zero, the
// previous step's solution (warm start, re-read from its FP64 copy), or the linear extrapolation
// 2 phi_{n-1} - phi_{n-2} of the last two (extrap, once two solves exist); the fixed point is the
// same whatever the start. It is written to phi_old (the first reduction's reference) and the
// sources are formed from it.
template <typename T>
__global__ void sn_source_kernel(int ncells, CellSplit split, int wave, Wave<T> wv, const T* sig, T* phi_old,
                                 const double* prev, const double* prev2, const DevState* st, int extrap,
                                 const double* mom, T area, T inv_4pi_dt, T inv_cdt, T* src, T* sgA) {
    pdl_wait();
    pdl_trigger();   // the first sweep may be scheduled now; it waits for this kernel before reading
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncells) return;
    int ix, iy;
    split(k, &ix, &iy);
    const int wst = st->sn_warm;
    T po[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const size_t e = 4 * (size_t)k + i;
        po[i] = wst == 0 ? T(0) : (extrap && wst >= 2 ? (T)(2.0 * prev[e] - prev2[e]) : (T)prev[e]);
        phi_old[e] = po[i];
    }
    const T sa = sig[2 * k], ss = sig[2 * k + 1];
    T S[4];
    source4<T>(ss, area, po, mom + 4 * (size_t)k, inv_4pi_dt, S);
    const T g = (sa + ss + inv_cdt) * area;
    size_t e[4];
    const int n = sweep_entries<T>(wave != 0, wv, split.nx, ix, iy, e);
    for (int j = 0; j < n; ++j) {
        T* d = src + 4 * e[j];
        d[0] = S[0]; d[1] = S[1]; d[2] = S[2]; d[3] = S[3];
        sgA[e[j]] = g;
    }
}

// source integral i of cell (ix, iy) into the sweep's entries
template <typename T>
__device__ __forceinline__ void put_source(T* src, bool wave, const Wave<T>& wv, int nx, int ix, int iy, int i, T v) {
    size_t e[4];
    const int n = sweep_entries<T>(wave, wv, nx, ix, iy, e);
    for (int j = 0; j < n; ++j) src[4 * e[j] + i] = v;
}

// Cell data of one wavefront step: the four source integrals (un-mirrored) and (sigma_t + 1/(c dt)) A.
template <typename T> struct CellIn { T s0, s1, s2, s3, sA; };

// s4: the cell's four source integrals, sa: its sigma* A (two arrays, so that the cells a lane takes
// in consecutive steps share sectors)
__device__ __forceinline__ void load_cell(const float* s4, const float* sa, CellIn<float>& d) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(s4));
    d.s0 = v.x; d.s1 = v.y; d.s2 = v.z; d.s3 = v.w;
    d.sA = __ldg(sa);
}
__device__ __forceinline__ void load_cell(const double* s4, const double* sa, CellIn<double>& d) {
    const double2 v0 = __ldg(reinterpret_cast<const double2*>(s4));
    const double2 v1 = __ldg(reinterpret_cast<const double2*>(s4) + 1);
    d.s0 = v0.x; d.s1 = v0.y; d.s2 = v1.x; d.s3 = v1.y;
    d.sA = __ldg(sa);
}

__device__ __forceinline__ void store_cell(float* d, float a0, float a1, float a2, float a3) {
    *reinterpret_cast<float4*>(d) = make_float4(a0, a1, a2, a3);
}
__device__ __forceinline__ void store_cell(double* d, double a0, double a1, double a2, double a3) {
    reinterpret_cast<double2*>(d)[0] = make_double2(a0, a1);
    reinterpret_cast<double2*>(d)[1] = make_double2(a2, a3);
}

// a predicated store of one cell's four coefficients (no branch in the step; an address formed for a
// lane that holds no cell is never accessed)
__device__ __forceinline__ void store_cell_if(bool p, float* d, float a0, float a1, float a2, float a3) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.global.v4.f32 [%1], {%2, %3, %4, %5};\n\t}"
        ::"r"((uint32_t)p), "l"(d), "f"(a0), "f"(a1), "f"(a2), "f"(a3)
        : "memory");
}
__device__ __forceinline__ void store_cell_if(bool p, double* d, double a0, double a1, double a2, double a3) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t"
        "@q st.global.v2.f64 [%1], {%2, %3};\n\t@q st.global.v2.f64 [%1+16], {%4, %5};\n\t}"
        ::"r"((uint32_t)p), "l"(d), "d"(a0), "d"(a1), "d"(a2), "d"(a3)
        : "memory");
}

// Strip-to-strip trace ring: each 32-bit piece of the two traces of a column travels with a 32-bit
// sequence tag in one 64-bit shared-memory word (a single-copy-atomic access; a vector store of
// such words is one access per word), so a reader that sees the expected tag in every word of the
// entry has the values, with no fence and no counter.
template <typename T> struct Ring;
template <> struct Ring<float> {
    static constexpr int kWords = 2;
    // stores the entry at shared address e when p (a predicated store: no branch in the step)
    static __device__ __forceinline__ void put_if(bool p, uint32_t e, float v0, float v1, uint32_t tag) {
        asm volatile(
            "{\n\t.reg .pred q;\n\t.reg .b64 w0, w1;\n\t"
            "setp.ne.u32 q, %0, 0;\n\t"
            "mov.b64 w0, {%2, %4};\n\tmov.b64 w1, {%3, %4};\n\t"
            "@q st.volatile.shared.v2.u64 [%1], {w0, w1};\n\t}"
            ::"r"((uint32_t)p), "r"(e), "r"(__float_as_uint(v0)), "r"(__float_as_uint(v1)), "r"(tag)
            : "memory");
    }
    // true when both words carry the tag; the values in v0, v1
    static __device__ __forceinline__ bool get(const volatile unsigned long long* e, uint32_t tag, float* v0, float* v1) {
        const unsigned long long a = e[0], b = e[1];
        *v0 = __uint_as_float((uint32_t)a);
        *v1 = __uint_as_float((uint32_t)b);
        return (uint32_t)(a >> 32) == tag && (uint32_t)(b >> 32) == tag;
    }
};
template <> struct Ring<double> {
    static constexpr int kWords = 4;
    static __device__ __forceinline__ void put_if(bool p, uint32_t e, double v0, double v1, uint32_t tag) {
        asm volatile(
            "{\n\t.reg .pred q;\n\t.reg .b64 w0, w1, w2, w3;\n\t"
            "setp.ne.u32 q, %0, 0;\n\t"
            "mov.b64 w0, {%2, %6};\n\tmov.b64 w1, {%3, %6};\n\t"
            "mov.b64 w2, {%4, %6};\n\tmov.b64 w3, {%5, %6};\n\t"
            "@q st.volatile.shared.v2.u64 [%1], {w0, w1};\n\t"
            "@q st.volatile.shared.v2.u64 [%1+16], {w2, w3};\n\t}"
            ::"r"((uint32_t)p), "r"(e), "r"((uint32_t)__double2loint(v0)), "r"((uint32_t)__double2hiint(v0)),
              "r"((uint32_t)__double2loint(v1)), "r"((uint32_t)__double2hiint(v1)), "r"(tag)
            : "memory");
    }
    static __device__ __forceinline__ bool get(const volatile unsigned long long* e, uint32_t tag, double* v0, double* v1) {
        const unsigned long long a = e[0], b = e[1], c = e[2], d = e[3];
        *v0 = __hiloint2double((int)(uint32_t)b, (int)(uint32_t)a);
        *v1 = __hiloint2double((int)(uint32_t)d, (int)(uint32_t)c);
        return (uint32_t)(a >> 32) == tag && (uint32_t)(b >> 32) == tag && (uint32_t)(c >> 32) == tag &&
               (uint32_t)(d >> 32) == tag;
    }
};

// reciprocals of the sweep's cell solve: FP32 takes the single-instruction approximation
// (relative error below 2^-22), FP64 the correctly rounded quotient
__device__ __forceinline__ float sweep_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double sweep_rcp(double x) { return 1.0 / x; }

// The mirrored cell system couples {a0, a3} only to {a1, a2}:
//   [ d0  2X  2Y   0 ]        d0 = sA + 2X + 2Y,       d1 = sA/3 + 2X + (2/3)Y,
//   [-2X  d1   0  tY ]        d2 = sA/3 + (2/3)X + 2Y, d3 = sA/9 + (2/3)(X + Y),
//   [-2Y   0  d2  tX ]        tX = (2/3)X, tY = (2/3)Y;
//   [  0 -tY -tX  d3 ]
// eliminating a0 and a3 leaves a symmetric positive 2x2 system for (a1, a2) (Schur complement).
// Per cell and ordinate, the coefficients that do not depend on the incoming traces are computed
// ahead, off the wavefront chain; with b the right-hand side,
//   r1 = b1 + k1 b0 - k2 b3,  r2 = b2 + k3 b0 - k4 b3,  a1 = Di r1 - Bi r2,  a2 = Ai r2 - Bi r1,
//   a0 = (b0 - 2X a1 - 2Y a2) i0,  a3 = (b3 + tY a1 + tX a2) i3.
template <typename T>
struct CellSolve { T k1, k2, k3, k4, Ai, Bi, Di, i0, i3; };

template <typename T>
__device__ __forceinline__ CellSolve<T> cell_solve(T sA, T X, T Y) {
    const T twoX = T(2) * X, twoY = T(2) * Y, tX = T(2.0 / 3.0) * X, tY = T(2.0 / 3.0) * Y;
    const T d0 = sA + twoX + twoY;
    const T d1 = sA * T(1.0 / 3.0) + twoX + tY;
    const T d2 = sA * T(1.0 / 3.0) + tX + twoY;
    const T d3 = sA * T(1.0 / 9.0) + tX + tY;
    CellSolve<T> c;
    c.i0 = sweep_rcp(d0);
    c.i3 = sweep_rcp(d3);
    const T A = d1 + twoX * twoX * c.i0 + tY * tY * c.i3;
    const T B = twoX * twoY * c.i0 + tX * tY * c.i3;
    const T D = d2 + twoY * twoY * c.i0 + tX * tX * c.i3;
    const T idet = sweep_rcp(A * D - B * B);
    c.k1 = twoX * c.i0; c.k2 = tY * c.i3; c.k3 = twoY * c.i0; c.k4 = tX * c.i3;
    c.Ai = A * idet; c.Bi = B * idet; c.Di = D * idet;
    return c;
}


// The cell-solve table: the mirrored cell system depends only on the cell's (sigma_t + 1/(c dt)) A
// and on |Omega_x|, |Omega_y|, which the four quadrants share, so per class q (the ordinates m with
// m mod nq = q) and padded cell it holds the nine coefficients of the solve (k1..k4, Ai, Bi, Di, i0
// in k8; i3). The cross sections are fixed for a problem's life, so it is built once; halo entries
// are zero, and a solve with zero coefficients returns zero. The expressions are the step's own,
// so the tabulated and the in-step solve agree bit for bit. Kept for FP64 only: there the step's
// three correctly rounded divisions on the FP64 pipe cost more than the table's loads (measured:
// the 6-iteration S8 solve on 112^2 cells 6.18 -> 2.94 ms), while FP32's approximate reciprocals
// cost less than the extra loads and registers (0.318 -> 0.380 ms with the table).
constexpr size_t kTableMaxBytes = size_t(32) << 20;   // kept only where it stays resident in L2
constexpr int kTableMaxStrips = 8;                    // the table sweep runs at most 8 warps per CTA

template <typename T>
__global__ void sn_table_kernel(int ncells, int nq, CellSplit split, const T* sig, T area, T inv_cdt, const T* qox,
                                const T* qoy, T dx, T dy, size_t plane, T* k8, T* i3) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)ncells * nq) return;
    const int q = (int)(e / ncells), k = (int)(e - (long long)q * ncells);
    int ix, iy;
    split(k, &ix, &iy);
    const size_t r = (size_t)q * plane + SweepPad<T>::at(split.nx, ix, iy);
    const T sa = sig[2 * k], ss = sig[2 * k + 1];
    const T sA = (sa + ss + inv_cdt) * area;
    const T X = fabs(qox[q]) * dy * T(0.5), Y = fabs(qoy[q]) * dx * T(0.5);
    const CellSolve<T> c = cell_solve<T>(sA, X, Y);
    T* o = k8 + r * 8;
    o[0] = c.k1; o[1] = c.k2; o[2] = c.k3; o[3] = c.k4;
    o[4] = c.Ai; o[5] = c.Bi; o[6] = c.Di; o[7] = c.i0;
    i3[r] = c.i3;
}

// Cell data of one wavefront step with the cell solve taken from the table.
template <typename T> struct CellInT { T s0, s1, s2, s3; CellSolve<T> cs; };

__device__ __forceinline__ void load_cell_tab(const float* s4, const float* k8, const float* i3, CellInT<float>& d) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(s4));
    const float4 a = __ldg(reinterpret_cast<const float4*>(k8));
    const float4 b = __ldg(reinterpret_cast<const float4*>(k8) + 1);
    d.s0 = v.x; d.s1 = v.y; d.s2 = v.z; d.s3 = v.w;
    d.cs.k1 = a.x; d.cs.k2 = a.y; d.cs.k3 = a.z; d.cs.k4 = a.w;
    d.cs.Ai = b.x; d.cs.Bi = b.y; d.cs.Di = b.z; d.cs.i0 = b.w;
    d.cs.i3 = __ldg(i3);
}
__device__ __forceinline__ void load_cell_tab(const double* s4, const double* k8, const double* i3, CellInT<double>& d) {
    const double2 v0 = __ldg(reinterpret_cast<const double2*>(s4));
    const double2 v1 = __ldg(reinterpret_cast<const double2*>(s4) + 1);
    const double2 a0 = __ldg(reinterpret_cast<const double2*>(k8));
    const double2 a1 = __ldg(reinterpret_cast<const double2*>(k8) + 1);
    const double2 b0 = __ldg(reinterpret_cast<const double2*>(k8) + 2);
    const double2 b1 = __ldg(reinterpret_cast<const double2*>(k8) + 3);
    d.s0 = v0.x; d.s1 = v0.y; d.s2 = v1.x; d.s3 = v1.y;
    d.cs.k1 = a0.x; d.cs.k2 = a0.y; d.cs.k3 = a1.x; d.cs.k4 = a1.y;
    d.cs.Ai = b0.x; d.cs.Bi = b0.y; d.cs.Di = b1.x; d.cs.i0 = b1.y;
    d.cs.i3 = __ldg(i3);
}

// Pipelined strip sweep of one ordinate, W warps, in coordinates mirrored to +x, +y (SX: the x
// direction of the ordinate before mirroring; the y mirror only changes a strip's first row). Warp w
// sweeps strips w, w+W, ... (lane = row, one anti-diagonal per step). The trace leaving the top row
// of strip s goes through entry (slot s mod W, step) of a tagged shared-memory ring to the first row
// of strip s+1; the reader waits until the entries of its next PF columns carry their sequence
// numbers. When strips outnumber the warps a slot is reused, and its writer first waits for the
// previous reader's consumed-column counter (published once per prefetch block). Every wait is
// bounded and records kStSegments on exhaustion. Dependencies only point to lower strips, and all
// warps of the CTA are resident, so the pipeline always advances. Between the waits a block of PF
// steps is straight-line code: addresses are the lane's base plus compile-time offsets on the padded
// mesh, the stores are predicated, and nothing is tested per step. TAB: the cell solve comes from the
// precomputed table instead of being formed in the step. WAVE: sources and psi in the wavefront order
// of the ordinate's direction (a step's accesses are coalesced runs, psi is stored unpredicated into
// entries that hold no cell).
template <typename T, int SX, bool TAB, bool WAVE>
__device__ __forceinline__ void sweep_ordinate(const SweepArgs<T>& a, int m, int sy, volatile int* cons,
                                               volatile unsigned long long* ring, uint32_t ring_sa,
                                               bool& timed_out) {
    constexpr int PF = SweepDepth<T>::value;
    constexpr int RW = Ring<T>::kWords;
    const int W = a.W;
    const int nx = a.nx, ny = a.ny, re = a.re;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T syf = (T)sy, sxy = (T)(SX * sy), sxf = (T)SX;
    const T X = fabs(a.qox[m]) * a.dy * T(0.5), Y = fabs(a.qoy[m]) * a.dx * T(0.5);
    const T twoX = T(2) * X, twoY = T(2) * Y, tX = T(2.0 / 3.0) * X, tY = T(2.0 / 3.0) * Y;
    // per-step strides (in T) of a lane's source, sigma* A and psi pointers
    constexpr long long SS = WAVE ? 128 : SX * 4, AS = WAVE ? 32 : SX, PS = WAVE ? 128 : SX * 4;
    const size_t wsz = a.wv.size();
    const int Q = m / a.nq;
    T* out = a.psi + (size_t)m * (WAVE ? wsz : (size_t)nx * ny) * 4;
    const int nstrip = (ny + 31) / 32;
    const bool reuse = nstrip > W;
    const int nsteps = nx + 31;
    for (int s = warp; s < nstrip && !timed_out; s += W) {
        const int ly = 32 * s + lane;
        const int iy = ly < ny ? (sy > 0 ? ly : ny - 1 - ly) : ny;   // rows past the mesh: the extra row
        // padded mesh: this lane's cell at step t is base + SX t (column t - lane in mirrored x);
        // wavefront order: entry e0 + 32 t of the direction's arrays
        const long long base = (long long)SweepPad<T>::at(nx, SX > 0 ? 0 : nx - 1, iy) - (long long)SX * lane;
        const size_t e0 = (size_t)Q * wsz + (size_t)s * a.wv.nt * 32 + lane;
        const T* src = WAVE ? a.src + e0 * 4 : a.src + base * 4;
        const T* sga = WAVE ? a.sgA + e0 : a.sgA + base;
        const size_t toff = TAB ? (size_t)(m % a.nq) * a.plane : 0;   // table rows of this ordinate's class
        const T* tk8 = TAB ? a.k8 + (toff + base) * 8 : nullptr;
        const T* ti3 = TAB ? a.i3 + toff + base : nullptr;
        // psi of this lane's cell at step t: po + PS t (on the plain mesh formed only where the lane
        // holds a cell)
        T* po = WAVE ? out + (e0 - (size_t)Q * wsz) * 4
                     : out + ((long long)iy * nx + (SX > 0 ? 0 : nx - 1) - (long long)SX * lane) * 4;
        const unsigned nxl = ly < ny ? (unsigned)nx : 0u;   // columns this lane stores (plain mesh)
        const int bin = (s - 1 + W) % W, bout = s % W;
        const int qin = ((s - 1) / W) * nx, qout = (s / W) * nx;   // sequence bases of the ring slots
        const bool has_in = s > 0, has_out = s + 1 < nstrip;
        const bool put = has_out && lane == 31;
        // the reader takes column t from entry t + 31; lane 31 writes column t - 31 into entry t
        volatile unsigned long long* rin = ring + (size_t)bin * re * RW;
        const uint32_t rout = ring_sa + (uint32_t)((size_t)bout * re * RW * 8);
        T bx0 = 0, bx1 = 0, oy0 = 0, oy1 = 0;
        typename std::conditional<TAB, CellInT<T>, CellIn<T>>::type q[PF];
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            if constexpr (TAB) load_cell_tab(src + SX * i * 4, tk8 + SX * i * 8, ti3 + SX * i, q[i]);
            else load_cell(src + SS * i, sga + AS * i, q[i]);
        }
        for (int t0 = 0; t0 < nsteps; t0 += PF) {
            // a reused slot: the previous reader must have taken the columns this block writes
            if (reuse && has_out && s >= W) {
                const int need = qout - nx + (t0 + PF - 31 < nx ? t0 + PF - 31 : nx);
                int spins = 0;
                while (cons[bout] < need) {
                    if (++spins > a.poll_limit) { timed_out = true; break; }
                    __nanosleep(20);
                }
            }
            // the incoming traces of this block's columns (lane 0's row), taken from the ring once all
            // carry their tags. Waiting once per block keeps the block's steps one straight-line
            // sequence, so the trace-independent cell solves of later steps fill the latency of the
            // current step's chain. Every lane reads the same entries (broadcast): the wait is uniform.
            T rv0[PF], rv1[PF];
#pragma unroll
            for (int i = 0; i < PF; ++i) { rv0[i] = T(0); rv1[i] = T(0); }
            if (has_in && t0 < nx) {
                int spins = 0;
                for (;;) {
                    bool ok = true;
#pragma unroll
                    for (int i = 0; i < PF; ++i) {
                        const int t = t0 + i;
                        if (t < nx) ok &= Ring<T>::get(rin + (size_t)(t + 31) * RW, (uint32_t)(qin + t + 1), &rv0[i], &rv1[i]);
                    }
                    if (ok) break;
                    if (++spins > a.poll_limit) { timed_out = true; break; }
                    __nanosleep(20);
                }
            }
            const T* sb = src + SS * (t0 + PF);
            const T* ab = sga + AS * (t0 + PF);
            const T* kb = TAB ? tk8 + (long long)SX * (t0 + PF) * 8 : nullptr;
            const T* jb = TAB ? ti3 + (long long)SX * (t0 + PF) : nullptr;
            T* pb = po + PS * t0;
            const uint32_t wb = rout + (uint32_t)(t0 * RW * 8);
            const uint32_t tagb = (uint32_t)(qout + t0 - 30);
#pragma unroll
            for (int i = 0; i < PF; ++i) {
                const T u0 = __shfl_up_sync(0xffffffffu, oy0, 1);
                const T u1 = __shfl_up_sync(0xffffffffu, oy1, 1);
                const T by0 = lane == 0 ? rv0[i] : u0;
                const T by1 = lane == 0 ? rv1[i] : u1;
                CellSolve<T> cs;
                if constexpr (TAB) cs = q[i].cs;
                else cs = cell_solve<T>(q[i].sA, X, Y);
                const T b0 = q[i].s0 + twoX * bx0 + twoY * by0;
                const T b1 = sxf * q[i].s1 - twoX * bx0 + tY * by1;
                const T b2 = syf * q[i].s2 + tX * bx1 - twoY * by0;
                const T b3 = sxy * q[i].s3 - tX * bx1 - tY * by1;
                const T r1 = b1 + cs.k1 * b0 - cs.k2 * b3;
                const T r2 = b2 + cs.k3 * b0 - cs.k4 * b3;
                const T a1 = cs.Di * r1 - cs.Bi * r2;
                const T a2 = cs.Ai * r2 - cs.Bi * r1;
                const T a0 = cs.i0 * b0 - cs.k1 * a1 - cs.k3 * a2;   // (b0 - 2X a1 - 2Y a2) / d0
                const T a3 = cs.i3 * b3 + cs.k2 * a1 + cs.k4 * a2;   // (b3 + tY a1 + tX a2) / d3
                bx0 = a0 + a1; bx1 = a2 + a3;
                oy0 = a0 + a2; oy1 = a1 + a3;
                if constexpr (WAVE) store_cell(pb + PS * i, a0, a1, a2, a3);
                else store_cell_if((unsigned)(t0 + i - lane) < nxl, pb + PS * i, a0, a1, a2, a3);
                Ring<T>::put_if(put, wb + (uint32_t)(i * RW * 8), oy0, oy1, tagb + (uint32_t)i);
                if constexpr (TAB) load_cell_tab(sb + SX * i * 4, kb + SX * i * 8, jb + SX * i, q[i]);
                else load_cell(sb + SS * i, ab + AS * i, q[i]);
            }
            // publish the columns this warp has taken from its input slot (only needed on reuse)
            if (reuse && has_in && lane == 0) {
                __threadfence_block();
                cons[bin] = qin + (t0 + PF < nx ? t0 + PF : nx);
            }
            if (__any_sync(0xffffffffu, timed_out)) { timed_out = true; break; }
        }
    }
}

template <typename T, bool TAB, bool WAVE>
__global__ void __launch_bounds__(TAB ? 256 : 512) sweep_pipe_kernel(SweepArgs<T> a) {
    static_assert(!(TAB && WAVE), "the cell-solve table is kept on the padded mesh only");
    constexpr int RW = Ring<T>::kWords;
    pdl_wait();
    pdl_trigger();
    if (*(volatile const int*)a.conv) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int W = a.W;
    volatile int* cons = (volatile int*)smraw;
    const size_t ring_off = ((W * sizeof(int) + 15) / 16) * 16;
    volatile unsigned long long* ring = (volatile unsigned long long*)(smraw + ring_off);   // W x re x RW
    for (int i = threadIdx.x; i < W; i += blockDim.x) cons[i] = 0;
    for (int i = threadIdx.x; i < W * a.re * RW; i += blockDim.x) ring[i] = 0ull;   // no tag is 0
    __syncthreads();
    const int m = blockIdx.x;
    const int quad = m / a.nq;
    const int sy = (quad <= 1) ? 1 : -1;
    const uint32_t ring_sa = (uint32_t)__cvta_generic_to_shared(smraw + ring_off);
    bool timed_out = false;
    if (quad == 0 || quad == 3) sweep_ordinate<T, 1, TAB, WAVE>(a, m, sy, cons, ring, ring_sa, timed_out);
    else sweep_ordinate<T, -1, TAB, WAVE>(a, m, sy, cons, ring, ring_sa, timed_out);
    if (timed_out && (threadIdx.x & 31) == 0) atomicOr(a.status, kStSegments);
}

// One source iteration's reduction. A block covers 32 cells: thread (g, c) sums the weighted
// ordinate solutions of cell c over ordinates g, g+8, ... (vector loads, coalesced across c); the
// 8 partials of a cell are added in g order in shared memory, then thread (c, i) forms coefficient
// i of phi_new, its contribution to the change norm and the next iteration's source integral i.
// The block's norm partials go to part[]; reduce_partials (below) adds them in a fixed order in
// the last block to finish, which applies the stop test
//   ||phi_new - phi_old|| <= tol ||phi_new||   (or no source at all),
// so the reduction and the test are one launch and the result does not depend on block order.
constexpr int kRedCells = 32, kRedGroups = 8;
constexpr int kRedThreads = kRedCells * kRedGroups;
constexpr int kRedGroupBlocks = kRedThreads;   // blocks per group of the two-level completion

// Sums NV values over the 256 threads of the block in a fixed tree (warp shuffles, then the 8 warp
// sums in warp order); thread q < NV receives total q.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sw)[kRedThreads / 32], double* out) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sw[q][threadIdx.x >> 5] = v[q];
    __syncthreads();
    if (threadIdx.x < NV) {
        double a = 0;
        for (int w = 0; w < kRedThreads / 32; ++w) a += sw[threadIdx.x][w];
        out[threadIdx.x] = a;
    }
}

// Two-level completion of per-block partial sums, independent of the order in which blocks finish.
// Block b has written its NV partials to part[b NV + q], each writing thread followed by a
// __threadfence (only those threads: a fence in every thread would also wait for the block's other
// stores); all threads call this after that.
// Every kRedGroupBlocks consecutive blocks form a group; the last block of a group to arrive adds
// the group's partials (one per thread, then block_sum) into gpart[g NV + q]; the last group to
// arrive adds the group sums (a fixed sequence per thread, then block_sum) into s_tot. Returns
// true in that one block, with the totals in s_tot (shared). The arrival counters gcnt[g] and
// *top reset themselves. Partials are re-read with volatile loads after the writers' fences.
template <int NV>
__device__ bool reduce_partials(double* part, int nblk, double* gpart, unsigned* gcnt, unsigned* top,
                                double* s_tot) {
    __shared__ double sw[NV][kRedThreads / 32];
    __shared__ bool s_go;
    const int g = blockIdx.x / kRedGroupBlocks;
    const int ngrp = (nblk + kRedGroupBlocks - 1) / kRedGroupBlocks;
    const int b0 = g * kRedGroupBlocks;
    const int gsize = nblk - b0 < kRedGroupBlocks ? nblk - b0 : kRedGroupBlocks;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_go = atomicAdd(&gcnt[g], 1u) == (unsigned)gsize - 1u;
    }
    __syncthreads();
    if (!s_go) return false;
    __threadfence();
    double v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q)
        v[q] = (int)threadIdx.x < gsize ? ((volatile double*)part)[(size_t)(b0 + threadIdx.x) * NV + q] : 0.0;
    block_sum<NV>(v, sw, s_tot);
    if (threadIdx.x < NV) {
        gpart[(size_t)g * NV + threadIdx.x] = s_tot[threadIdx.x];
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        gcnt[g] = 0u;
        s_go = atomicAdd(top, 1u) == (unsigned)ngrp - 1u;
    }
    __syncthreads();
    if (!s_go) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = 0.0;
    for (int j = threadIdx.x; j < ngrp; j += kRedThreads)
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] += ((volatile double*)gpart)[(size_t)j * NV + q];
    __syncthreads();
    block_sum<NV>(v, sw, s_tot);
    if (threadIdx.x == 0) *top = 0u;
    __syncthreads();
    return true;
}

// Scratch of the source-iteration reductions inside the sn_norm buffer: block partials (up to
// kAAMax + 2 per block), group partials, group arrival counters.
struct RedScratch {
    double* part;
    double* gpart;
    unsigned* gcnt;
};
constexpr int kAAMax = 8;   // deepest Anderson history

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    static __device__ __forceinline__ void load(const float* p, float* v) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    }
};
template <> struct Vec4<double> {
    static __device__ __forceinline__ void load(const double* p, double* v) {
        const double2 x = reinterpret_cast<const double2*>(p)[0], y = reinterpret_cast<const double2*>(p)[1];
        v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
    }
};

// The ordinate sum of one cell over ordinates g, g + kRedGroups, ...: psi_m (mirrored coefficients;
// plain mesh, or the cell's entry in the wavefront order of m's quadrant) times the signed weights
// (w_m, w_m s_x, w_m s_y, w_m s_x s_y) that undo the mirror, in ordinate order.
template <typename T>
__device__ __forceinline__ void weighted_psi_sum(const T* psi, int nord, int nq, bool wave, const Wave<T>& wv,
                                                 CellSplit split, const T* qwv, int k, int ncells, int g, T* out) {
    constexpr int kPer = (kMaxOrd + kRedGroups - 1) / kRedGroups;   // ordinates per thread, at most
    T acc[4] = {0, 0, 0, 0};
    if (k < ncells) {
        size_t e[4] = {(size_t)k, (size_t)k, (size_t)k, (size_t)k};   // per quadrant: entry of the cell
        size_t plane = (size_t)ncells;
        if (wave) {
            int ix, iy;
            split(k, &ix, &iy);
#pragma unroll
            for (int Q = 0; Q < 4; ++Q) e[Q] = wv.at(ix, iy, quad_sx(Q), quad_sy(Q));
            plane = wv.size();
        }
        // all loads first (in flight together), then the sum in ordinate order
        T v[kPer][4];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int m = g + j * kRedGroups;
            if (m < nord) {
                const int Q = (m >= nq) + (m >= 2 * nq) + (m >= 3 * nq);
                Vec4<T>::load(psi + ((size_t)m * plane + e[Q]) * 4, v[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int m = g + j * kRedGroups;
            if (m < nord) {
                T w[4];
                Vec4<T>::load(qwv + 4 * m, w);
                acc[0] += w[0] * v[j][0]; acc[1] += w[1] * v[j][1]; acc[2] += w[2] * v[j][2]; acc[3] += w[3] * v[j][3];
            }
        }
    }
    out[0] = acc[0]; out[1] = acc[1]; out[2] = acc[2]; out[3] = acc[3];
}

template <typename T>
__global__ void __launch_bounds__(kRedCells * kRedGroups)
sn_reduce_kernel(const T* psi, int nord, int nq, int wave, Wave<T> wv, const T* qwv, CellSplit split, const T* phi_old,
                 T* phi_new,
                 int ncells, RedScratch rs, const T* sig, const double* mom, T area, T inv_4pi_dt, T* src, DevState* st,
                 double tol) {
    __shared__ T sp[kRedGroups][kRedCells][4];
    __shared__ double sred[2][kRedCells * 4 / 32];
    __shared__ double s_tot[2];
    const int c = threadIdx.x % kRedCells, g = threadIdx.x / kRedCells;
    const int k0 = blockIdx.x * kRedCells;
    pdl_wait();
    if (*(volatile const int*)&st->sn_conv) {
        pdl_trigger();
        // converged earlier: carry the solution forward so the buffer alternation stays aligned
        if (threadIdx.x < kRedCells * 4) {
            const size_t e = (size_t)k0 * 4 + threadIdx.x;
            if (e < (size_t)ncells * 4) phi_new[e] = phi_old[e];
        }
        return;
    }
    weighted_psi_sum<T>(psi, nord, nq, wave != 0, wv, split, qwv, k0 + c, ncells, g, sp[g][c]);
    __syncthreads();
    if (threadIdx.x < kRedCells * 4) {
        const int cc = threadIdx.x >> 2, i = threadIdx.x & 3;
        const int k = k0 + cc;
        T num = 0, den = 0;
        if (k < ncells) {
            T v = 0;
#pragma unroll
            for (int q = 0; q < kRedGroups; ++q) v += sp[q][cc][i];
            const size_t e = (size_t)k * 4 + i;
            phi_new[e] = v;
            const T nrm = i == 0 ? T(1) : (i == 3 ? T(1.0 / 9.0) : T(1.0 / 3.0));
            const T n_i = nrm;   // the Legendre norm of coefficient i is the same factor
            const T d = v - phi_old[e];
            num = nrm * d * d;
            den = nrm * v * v;
            // source integral i: sigma_s A n_i phi_i / (4 pi) + m_i / (4 pi dt)
            const T cs = sig[2 * (size_t)k + 1] * area * T(0.07957747154594767);
            int ix, iy;
            split(k, &ix, &iy);
            put_source<T>(src, wave != 0, wv, split.nx, ix, iy, i, cs * v * n_i + (T)mom[e] * inv_4pi_dt);
        }
        // warp sums (fixed tree), then block sum in warp order
        for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_down_sync(0xffffffffu, num, o);
            den += __shfl_down_sync(0xffffffffu, den, o);
        }
        if ((threadIdx.x & 31) == 0) { sred[0][threadIdx.x >> 5] = (double)num; sred[1][threadIdx.x >> 5] = (double)den; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int q = 0; q < kRedCells * 4 / 32; ++q) { a += sred[0][q]; b += sred[1][q]; }
        rs.part[2 * blockIdx.x] = a;
        rs.part[2 * blockIdx.x + 1] = b;
        __threadfence();
    }
    pdl_trigger();   // late: the next sweep is scheduled as this reduction completes
    if (reduce_partials<2>(rs.part, (int)gridDim.x, rs.gpart, rs.gcnt, &st->sn_blocks_done, s_tot) &&
        threadIdx.x == 0) {
        const double a = s_tot[0], b = s_tot[1];
        st->sn_norm_num = a;
        st->sn_norm_den = b;
        st->sn_iters += 1;
        if (b == 0.0 || sqrt(a) <= tol * sqrt(b)) st->sn_conv = 1;
    }
}

// ---------------------------------------------------------------------------------------------
// Anderson acceleration of the source iteration (optional, depth 1..kAAMax). With G the
// iteration map (source -> sweep -> ordinate sum), g_k = G(phi_k) and residual f_k = g_k - phi_k,
// the next iterate is phi_{k+1} = sum_j alpha_j g_j over the last n stored iterates, alpha
// minimising || sum_j alpha_j f_j || with sum_j alpha_j = 1 (weighted L2 norm of the bilinear
// fields, as in the stop test). A fixed point of the map is a fixed point of the mixed
// iteration, so the converged flux is the plain iteration's; the stop test is the same
// ||f_k|| <= tol ||g_k||, and a converged solve returns g_k.
// ---------------------------------------------------------------------------------------------
struct AAState {
    int n, head, ok, pad;                     // stored iterates, next slot, mixing weights valid
    double gram[kAAMax + 1][kAAMax + 1];      // <f_s, f_t> over stored slots
    double alpha[kAAMax + 1];                 // mixing weights by slot (0 for empty slots)
};
constexpr int kAAPart = kAAMax + 2;           // per reduction block: dots with every slot, then <g, g>

// The constrained least squares of the mixing weights over the n valid slots (one thread):
// (G + eps I) y = 1, alpha = y / sum y, by elimination with partial pivoting.
__device__ void aa_solve(AAState* aa, const int* slots, int n) {
    double G[kAAMax + 1][kAAMax + 2];
    double dmax = 0;
    for (int a = 0; a < n; ++a) dmax = fmax(dmax, aa->gram[slots[a]][slots[a]]);
    for (int a = 0; a < n; ++a) {
        for (int b = 0; b < n; ++b) G[a][b] = aa->gram[slots[a]][slots[b]];
        G[a][a] += 1e-12 * dmax;
        G[a][n] = 1.0;
    }
    bool ok = dmax > 0;
    for (int c = 0; c < n && ok; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(G[r][c]) > fabs(G[piv][c])) piv = r;
        if (!(fabs(G[piv][c]) > 0)) { ok = false; break; }
        if (piv != c)
            for (int q = c; q <= n; ++q) { const double t = G[c][q]; G[c][q] = G[piv][q]; G[piv][q] = t; }
        for (int r = c + 1; r < n; ++r) {
            const double f = G[r][c] / G[c][c];
            for (int q = c; q <= n; ++q) G[r][q] -= f * G[c][q];
        }
    }
    double y[kAAMax + 1];
    double sy = 0;
    for (int r = n - 1; r >= 0 && ok; --r) {
        double v = G[r][n];
        for (int q = r + 1; q < n; ++q) v -= G[r][q] * y[q];
        y[r] = v / G[r][r];
        sy += y[r];
    }
    ok = ok && isfinite(sy) && fabs(sy) > 1e-300;
    for (int q = 0; q <= kAAMax; ++q) aa->alpha[q] = 0.0;
    if (ok)
        for (int a = 0; a < n; ++a) aa->alpha[slots[a]] = y[a] / sy;
    aa->ok = ok ? 1 : 0;
}

// The reduction of an accelerated iteration: g = sum of w_m psi_m (into phi_new and the history),
// f = g - phi_old, the weighted dots of f with every stored residual and <g, g>; the last block
// completes the Gram matrix, applies the stop test and, if the solve goes on, forms the weights.
template <typename T, int NS>
__global__ void __launch_bounds__(kRedCells * kRedGroups)
sn_reduce_aa_kernel(const T* psi, int nord, int nq, int wave, Wave<T> wv, CellSplit split, const T* qwv, const T* phi_old, T* phi_new,
                    int ncells, RedScratch rs, T* g_hist, T* f_hist, int depth, AAState* aa, DevState* st, double tol) {
    constexpr int NP = NS + 1;   // per block: the dots with the NS slots, then <g, g>
    __shared__ T sp[kRedGroups][kRedCells][4];
    __shared__ double sred[NP][kRedCells * 4 / 32];
    __shared__ double s_tot[NP];
    const int c = threadIdx.x % kRedCells, g = threadIdx.x / kRedCells;
    const int k0 = blockIdx.x * kRedCells;
    pdl_wait();
    if (*(volatile const int*)&st->sn_conv) {
        pdl_trigger();
        if (threadIdx.x < kRedCells * 4) {
            const size_t e = (size_t)k0 * 4 + threadIdx.x;
            if (e < (size_t)ncells * 4) phi_new[e] = phi_old[e];
        }
        return;
    }
    const int nslot = NS;   // depth + 1
    const int head = aa->head, n_new = aa->n + 1 < nslot ? aa->n + 1 : nslot;
    const size_t nv = (size_t)ncells * 4;
    weighted_psi_sum<T>(psi, nord, nq, wave != 0, wv, split, qwv, k0 + c, ncells, g, sp[g][c]);
    __syncthreads();
    if (threadIdx.x < kRedCells * 4) {
        const int cc = threadIdx.x >> 2, i = threadIdx.x & 3;
        const int k = k0 + cc;
        T dots[NS];
        T den = 0;
#pragma unroll
        for (int q = 0; q < NS; ++q) dots[q] = 0;
        if (k < ncells) {
            T v = 0;
#pragma unroll
            for (int q = 0; q < kRedGroups; ++q) v += sp[q][cc][i];
            const size_t e = (size_t)k * 4 + i;
            const T nrm = i == 0 ? T(1) : (i == 3 ? T(1.0 / 9.0) : T(1.0 / 3.0));
            const T f = v - phi_old[e];
            phi_new[e] = v;
            g_hist[head * nv + e] = v;
            f_hist[head * nv + e] = f;
            den = nrm * v * v;
            // the stored slots: head and the n_new - 1 before it in ring order
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const int j = (head - q + nslot) % nslot;
                if (j < n_new) dots[q] = nrm * f * (q == head ? f : f_hist[q * nv + e]);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            den += __shfl_down_sync(0xffffffffu, den, o);
#pragma unroll
            for (int q = 0; q < NS; ++q) dots[q] += __shfl_down_sync(0xffffffffu, dots[q], o);
        }
        if ((threadIdx.x & 31) == 0) {
            const int w = threadIdx.x >> 5;
#pragma unroll
            for (int q = 0; q < NS; ++q) sred[q][w] = (double)dots[q];
            sred[NS][w] = (double)den;
        }
    }
    __syncthreads();
    if (threadIdx.x < NP) {
        double a = 0;
        for (int w = 0; w < kRedCells * 4 / 32; ++w) a += sred[threadIdx.x][w];
        rs.part[(size_t)blockIdx.x * NP + threadIdx.x] = a;
        __threadfence();
    }
    pdl_trigger();   // late: the next sweep is scheduled as this reduction completes
    if (reduce_partials<NP>(rs.part, (int)gridDim.x, rs.gpart, rs.gcnt, &st->sn_blocks_done, s_tot) &&
        threadIdx.x == 0) {
        int slots[kAAMax + 1];
        for (int j = 0; j < n_new; ++j) {
            const int sl = (head - j + nslot) % nslot;
            slots[j] = sl;
            aa->gram[head][sl] = s_tot[sl];
            aa->gram[sl][head] = s_tot[sl];
        }
        const double num = s_tot[head], d = s_tot[NS];
        st->sn_norm_num = num;
        st->sn_norm_den = d;
        st->sn_iters += 1;
        if (d == 0.0 || sqrt(num) <= tol * sqrt(d)) st->sn_conv = 1;
        else aa_solve(aa, slots, n_new);
        aa->n = n_new;
        aa->head = (head + 1) % nslot;
    }
}

// The mixed iterate phi_{k+1} = sum alpha_s g_s (plain step g when the weights failed) and the
// source integrals of the next sweep from it.
template <typename T>
__global__ void sn_mix_kernel(T* phi_new, const T* g_hist, int ncells, int depth, const AAState* aa,
                              const DevState* st, const T* sig, const double* mom, T area, T inv_4pi_dt,
                              CellSplit split, int wave, Wave<T> wv, T* src) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nv = (size_t)ncells * 4;
    if (e >= nv || *(volatile const int*)&st->sn_conv) return;
    T v = phi_new[e];
    if (aa->ok) {
        double acc = 0;
        for (int q = 0; q <= depth; ++q) {
            const double al = aa->alpha[q];
            if (al != 0.0) acc += al * (double)g_hist[q * nv + e];
        }
        v = (T)acc;
        phi_new[e] = v;
    }
    const int i = (int)(e & 3);
    const size_t k = e >> 2;
    const T n_i = i == 0 ? T(1) : (i == 3 ? T(1.0 / 9.0) : T(1.0 / 3.0));
    const T cs = sig[2 * k + 1] * area * T(0.07957747154594767);
    int ix, iy;
    split((int)k, &ix, &iy);
    put_source<T>(src, wave != 0, wv, split.nx, ix, iy, i, cs * v * n_i + (T)mom[e] * inv_4pi_dt);
}

// The end of a solve: the solution's FP64 copy (with an extrapolating warm start, the copy it
// replaces moves to out_prev), the step flux phi_pre + phi_post + phi_c0 per cell, and the count
// of finished solves with warm starts enabled (up to 2), in one launch.
template <typename T>
__global__ void sn_finish_kernel(const T* phi, double* out, double* out_prev, int n, const double* pre,
                                 const double* post, double* flux, DevState* st, int warm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) st->sn_warm = warm ? min(st->sn_warm + 1, 2) : 0;
    if (i >= n) return;
    if (out_prev) out_prev[i] = out[i];
    const double v = (double)phi[i];
    out[i] = v;
    if ((i & 3) == 0) flux[i >> 2] = pre[i >> 2] + post[i >> 2] + v;
}

// the sn_norm buffer: kAAPart partials per reduction block, then per group, then the group counters
static RedScratch red_scratch(const hyb_problem* p) {
    const size_t nblk = (p->ncells + kRedCells - 1) / kRedCells;
    const size_t ngrp = (nblk + kRedGroupBlocks - 1) / kRedGroupBlocks;
    RedScratch r;
    r.part = p->sn_norm;
    r.gpart = r.part + kAAPart * nblk;
    r.gcnt = (unsigned*)(r.gpart + kAAPart * ngrp);
    return r;
}

size_t sn_norm_bytes(int ncells) {
    const size_t nblk = ((size_t)ncells + kRedCells - 1) / kRedCells;
    const size_t ngrp = (nblk + kRedGroupBlocks - 1) / kRedGroupBlocks;
    return kAAPart * (nblk + ngrp) * sizeof(double) + ngrp * sizeof(unsigned);
}

cudaError_t sn_clear_counters(hyb_problem* p) {
    const RedScratch r = red_scratch(p);
    const size_t nblk = (p->ncells + kRedCells - 1) / kRedCells;
    const size_t ngrp = (nblk + kRedGroupBlocks - 1) / kRedGroupBlocks;
    return cudaMemsetAsync(r.gcnt, 0, ngrp * sizeof(unsigned), p->stream);
}

template <typename T>
static size_t src_entries(int nx, int ny, int nord, int layout) {
    return sn_wave_layout(nx, ny, nord, sizeof(T) == 8, layout) ? 4 * Wave<T>::make(nx, ny).size()
                                                                 : SweepPad<T>::plane(nx, ny);
}

size_t sn_src_bytes(int nx, int ny, int nord, bool fp64, int layout) {
    return fp64 ? src_entries<double>(nx, ny, nord, layout) * 5 * sizeof(double)
                : src_entries<float>(nx, ny, nord, layout) * 5 * sizeof(float);
}

size_t sn_psi_bytes(int nx, int ny, int nord, bool fp64, int layout) {
    const size_t per = sn_wave_layout(nx, ny, nord, fp64, layout)
                           ? (fp64 ? Wave<double>::make(nx, ny).size() : Wave<float>::make(nx, ny).size())
                           : (size_t)nx * ny;
    return (size_t)nord * per * 4 * (fp64 ? 8 : 4);
}

// ring entries per slot: every step of a strip's last block, lane 31 trailing lane 0 by 31 columns
template <typename T>
static int ring_entries(int nx) { return nx + 31 + SweepDepth<T>::value; }

template <typename T>
static int sweep_warps(const hyb_problem* p, size_t* smem) {
    const int nstrip = (p->ny + 31) / 32;
    const size_t per = (size_t)ring_entries<T>(p->nx) * Ring<T>::kWords * sizeof(unsigned long long);
    int W = nstrip < 16 ? nstrip : 16;
    while (W > 1 && (size_t)W * per + 256 > 160 * 1024) --W;
    *smem = ((W * sizeof(int) + 15) / 16) * 16 + (size_t)W * per;
    return W;
}

template <typename T>
static cudaError_t sn_iteration_t(hyb_problem* p, int first) {
    cudaStream_t s = p->stream;
    const int g = (p->ncells + 255) / 256;
    const size_t plane = SweepPad<T>::plane(p->nx, p->ny);
    const int wave = sn_wave_layout(p->nx, p->ny, p->n_ord, sizeof(T) == 8, p->d.sn_layout) ? 1 : 0;
    const Wave<T> wv = Wave<T>::make(p->nx, p->ny);
    T* src = (T*)p->sn_quad;                                // 4 per entry
    T* sgA = src + 4 * src_entries<T>(p->nx, p->ny, p->n_ord, p->d.sn_layout);   // 1 per entry
    const CellSplit split = make_cell_split(p->nx);
    const int nq = p->n_ord / 4;
    const T inv4pidt = (T)(1.0 / (4.0 * 3.14159265358979323846 * p->d.dt));
    if (first)
        sn_source_kernel<T><<<g, 256, 0, s>>>(p->ncells, split, wave, wv, (const T*)p->sig, (T*)p->sn_phi_old,
                                              p->sn_phi_d, p->sn_phi_d2, p->st, p->d.sn_warm_start == 2 ? 1 : 0,
                                              p->mom_d, (T)p->area, inv4pidt, (T)(1.0 / (p->d.c * p->d.dt)), src,
                                              sgA);
    const T* qbuf = (const T*)p->sn_quadbuf;
    const T* qwv = qbuf + 3 * kMaxOrd;
    SweepArgs<T> a;
    a.nx = p->nx; a.ny = p->ny;
    a.nq = p->n_ord / 4;
    a.nord = p->n_ord;
    a.re = ring_entries<T>(p->nx);
    a.dx = (T)p->dx; a.dy = (T)p->dy;
    a.src = src;
    a.sgA = sgA;
    a.qox = qbuf; a.qoy = qbuf + kMaxOrd;
    a.psi = (T*)p->sn_psi;
    a.status = &p->st->status;
    a.poll_limit = p->d.wait_limit > 0 ? p->d.wait_limit : (1 << 22);
    a.conv = &p->st->sn_conv;
    a.plane = plane;
    a.wv = wv;
    size_t smem = 0;
    a.W = sweep_warps<T>(p, &smem);
    const bool tab = p->sn_table != nullptr && a.W <= kTableMaxStrips && !wave;
    a.k8 = tab ? (const T*)p->sn_table : nullptr;
    a.i3 = tab ? a.k8 + (size_t)a.nq * plane * 8 : nullptr;
    auto kern = wave ? sweep_pipe_kernel<T, false, true>
                     : (tab ? sweep_pipe_kernel<T, true, false> : sweep_pipe_kernel<T, false, false>);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaError_t le = launch_pdl(p->pdl, kern, dim3(p->n_ord), dim3(32 * a.W), smem, s, a);
    if (le != cudaSuccess) return le;
    const int gr = (p->ncells + kRedCells - 1) / kRedCells;
    const RedScratch rs = red_scratch(p);
    if (p->d.sn_accel > 0) {
        const int depth = p->d.sn_accel;
        const size_t nv = 4 * (size_t)p->ncells;
        T* gh = (T*)p->aa_hist;
        T* fh = gh + (size_t)(depth + 1) * nv;
        // the reduction carries depth + 2 partial sums per block: one instance per depth
        auto red = depth == 1 ? sn_reduce_aa_kernel<T, 2> : depth == 2 ? sn_reduce_aa_kernel<T, 3>
                 : depth == 3 ? sn_reduce_aa_kernel<T, 4> : depth == 4 ? sn_reduce_aa_kernel<T, 5>
                 : depth == 5 ? sn_reduce_aa_kernel<T, 6> : depth == 6 ? sn_reduce_aa_kernel<T, 7>
                 : depth == 7 ? sn_reduce_aa_kernel<T, 8> : sn_reduce_aa_kernel<T, 9>;
        le = launch_pdl(p->pdl, red, dim3(gr), dim3(kRedCells * kRedGroups), 0, s, (const T*)p->sn_psi, p->n_ord, nq, wave, wv,
                        split, qwv, (const T*)p->sn_phi_old, (T*)p->sn_phi, p->ncells, rs, gh, fh, depth,
                        (AAState*)p->aa_state, p->st, sn_tol_eff(p));
        if (le != cudaSuccess) return le;
        sn_mix_kernel<T><<<(unsigned)((nv + 255) / 256), 256, 0, s>>>((T*)p->sn_phi, gh, p->ncells, depth,
                                                                      (const AAState*)p->aa_state, p->st,
                                                                      (const T*)p->sig, p->mom_d, (T)p->area,
                                                                      inv4pidt, split, wave, wv, src);
        return cudaGetLastError();
    }
    le = launch_pdl(p->pdl, sn_reduce_kernel<T>, dim3(gr), dim3(kRedCells * kRedGroups), 0, s, (const T*)p->sn_psi, p->n_ord,
                    nq, wave, wv, qwv, split, (const T*)p->sn_phi_old, (T*)p->sn_phi, p->ncells, rs, (const T*)p->sig,
                    p->mom_d, (T)p->area, inv4pidt, src, p->st, sn_tol_eff(p));
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}

size_t sn_table_bytes(int nx, int ny, int nord, bool fp64, int layout) {
    if (!fp64 || (ny + 31) / 32 > kTableMaxStrips || sn_wave_layout(nx, ny, nord, fp64, layout)) return 0;
    const size_t b = fp64 ? (size_t)(nord / 4) * SweepPad<double>::plane(nx, ny) * 9 * sizeof(double)
                          : (size_t)(nord / 4) * SweepPad<float>::plane(nx, ny) * 9 * sizeof(float);
    return b <= kTableMaxBytes ? b : 0;
}

template <typename T>
static cudaError_t sn_build_table_t(hyb_problem* p) {
    const size_t plane = SweepPad<T>::plane(p->nx, p->ny);
    const int nq = p->n_ord / 4;
    T* k8 = (T*)p->sn_table;
    T* i3 = k8 + (size_t)nq * plane * 8;
    cudaError_t e = cudaMemsetAsync(p->sn_table, 0, (size_t)nq * plane * 9 * sizeof(T), p->stream);
    if (e != cudaSuccess) return e;
    const T* qbuf = (const T*)p->sn_quadbuf;
    const long long n = (long long)p->ncells * nq;
    sn_table_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(
        p->ncells, nq, make_cell_split(p->nx), (const T*)p->sig, (T)p->area, (T)(1.0 / (p->d.c * p->d.dt)), qbuf,
        qbuf + kMaxOrd, (T)p->dx, (T)p->dy, plane, k8, i3);
    return cudaGetLastError();
}

cudaError_t sn_build_table(hyb_problem* p) {
    if (!p->sn_table) return cudaSuccess;
    return p->prec == HYB_FP64 ? sn_build_table_t<double>(p) : sn_build_table_t<float>(p);
}

size_t sn_accel_state_bytes() { return sizeof(AAState); }

cudaError_t sn_start(hyb_problem* p) {
    cudaError_t e = cudaMemsetAsync(&p->st->sn_conv, 0, 2 * sizeof(int), p->stream);
    if (e != cudaSuccess) return e;
    if (p->d.sn_accel > 0) {   // an empty history for this solve
        e = cudaMemsetAsync(p->aa_state, 0, sizeof(AAState), p->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;   // the starting iterate is formed by the first iteration's source kernel
}

cudaError_t sn_iteration(hyb_problem* p, int first) {
    cudaError_t e = p->prec == HYB_FP64 ? sn_iteration_t<double>(p, first) : sn_iteration_t<float>(p, first);
    if (e != cudaSuccess) return e;
    void* t = p->sn_phi; p->sn_phi = p->sn_phi_old; p->sn_phi_old = t;   // newest is now sn_phi_old
    return cudaSuccess;
}

cudaError_t sn_finish(hyb_problem* p) {
    const int n = 4 * p->ncells;
    double* keep = p->d.sn_warm_start == 2 ? p->sn_phi_d2 : nullptr;
    const int warm = p->d.sn_warm_start ? 1 : 0;
    if (p->prec == HYB_FP64)
        sn_finish_kernel<double><<<(n + 255) / 256, 256, 0, p->stream>>>(
            (const double*)p->sn_phi_old, p->sn_phi_d, keep, n, p->pre_d, p->post_d, p->flux_d, p->st, warm);
    else
        sn_finish_kernel<float><<<(n + 255) / 256, 256, 0, p->stream>>>(
            (const float*)p->sn_phi_old, p->sn_phi_d, keep, n, p->pre_d, p->post_d, p->flux_d, p->st, warm);
    return cudaGetLastError();
}

}  // namespace hyb
