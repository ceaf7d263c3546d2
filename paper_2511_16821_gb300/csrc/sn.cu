// sn.cu -- collided S_N-DG stage (Sec. 2.2 step 2, Eq. (floor N_s+1)) on sm_103a.
//
// Backward Euler from zero data with vacuum boundaries:
//   (sigma_t + 1/(c dt)) Psi_c + Omega.grad Psi_c = (sigma_s / 4 pi)(phi_c + phi_{N_s}),
// where the fixed part comes from the hand-off moments m_i = sigma_s sum w int P_i ds (space-time
// integrals, so the source integral against P_i is m_i / (4 pi dt)). Bilinear DG per cell,
// psi = a0 + a1 xi + a2 eta + a3 xi eta, upwind traces, level-symmetric quadrature; source
// iteration on phi_c.
//
// Sweep: every ordinate of a quadrant shares one dependency order, so one CTA sweeps a 32x32 tile
// for all ordinates of its quadrant (thread = (tile row, ordinate), cells along the row in
// registers, the row-to-row trace through shared memory, one anti-diagonal per step). Tiles on
// one tile anti-diagonal run concurrently (one launch per tile anti-diagonal, the four quadrants in
// the same launch). Coordinates are mirrored per quadrant so that each sweep runs towards +x,+y;
// in mirrored coordinates the 4x4 cell system is the same for every quadrant and is diagonally
// dominant, so it is solved by elimination without pivoting.
#include <cuda_runtime.h>

#include <cmath>

#include "hyb_device.cuh"

namespace hyb {

template <typename T>
struct SweepArgs {
    int nx, ny, ntx, nty, nq, diag;
    T dx, dy, area, inv_cdt;
    const T* sig;            // (sigma_a, sigma_s) per cell
    const T* phi_old;        // 4 per cell
    const double* mom;       // hand-off moments, 4 per cell
    T inv_4pi_dt;
    const T* qox; const T* qoy; const T* qw;   // ordinates by quadrant: m = quad * nq + q
    T* phi_quad;             // 4 quadrants x ncells x 4
    T* tx;                   // outgoing x traces at tile columns: nord x ny x ntx x 2
    T* ty;                   // outgoing y traces at tile rows:    nord x nx x nty x 2
};

template <typename T>
__device__ __forceinline__ void solve4(T m[4][4], T b[4], T x[4]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int r = c + 1; r < 4; ++r) {
            const T f = m[r][c] / m[c][c];
#pragma unroll
            for (int k = c; k < 4; ++k) m[r][k] -= f * m[c][k];
            b[r] -= f * b[c];
        }
    }
#pragma unroll
    for (int r = 3; r >= 0; --r) {
        T s = b[r];
#pragma unroll
        for (int k = r + 1; k < 4; ++k) s -= m[r][k] * x[k];
        x[r] = s / m[r][r];
    }
}

template <typename T>
__global__ void sweep_tile_kernel(SweepArgs<T> a) {
    extern __shared__ unsigned char smraw[];
    T* ytr = (T*)smraw;                       // [nq][32][2]: y trace entering row r+1
    T* acc = ytr + a.nq * kSnTile * 2;        // [nq][32][4]: weighted psi of the step
    const int quad = blockIdx.y;
    const int sx = (quad == 0 || quad == 3) ? 1 : -1;
    const int sy = (quad <= 1) ? 1 : -1;
    const int tlx = max(0, a.diag - (a.nty - 1)) + blockIdx.x;
    const int tly = a.diag - tlx;
    if (tlx >= a.ntx || tly < 0 || tly >= a.nty) return;
    const int q = threadIdx.x / kSnTile, r = threadIdx.x % kSnTile;
    const int m = quad * a.nq + q;
    const T ox = a.qox[m], oy = a.qoy[m], wq = a.qw[m];
    const T X = fabs(ox) * a.dy * T(0.5), Y = fabs(oy) * a.dx * T(0.5);
    const int lx0 = tlx * kSnTile, ly0 = tly * kSnTile;
    const int ncx = min(kSnTile, a.nx - lx0), ncy = min(kSnTile, a.ny - ly0);
    const int ly = ly0 + r;
    const bool row_ok = r < ncy;
    const int iy = sy > 0 ? ly : a.ny - 1 - ly;
    // incoming x trace of this row (from the tile to the left, or vacuum)
    T bx0 = 0, bx1 = 0;
    if (row_ok && tlx > 0) {
        const T* s = a.tx + (((size_t)m * a.ny + ly) * a.ntx + (tlx - 1)) * 2;
        bx0 = s[0]; bx1 = s[1];
    }
    // incoming y traces of the tile's bottom row (from the tile below, or vacuum)
    for (int c = r; c < kSnTile; c += kSnTile) {
        T v0 = 0, v1 = 0;
        if (c < ncx && tly > 0) {
            const T* s = a.ty + (((size_t)m * a.nx + (lx0 + c)) * a.nty + (tly - 1)) * 2;
            v0 = s[0]; v1 = s[1];
        }
        ytr[(q * kSnTile + c) * 2] = v0;
        ytr[(q * kSnTile + c) * 2 + 1] = v1;
    }
    __syncthreads();
    const T sxf = (T)sx, syf = (T)sy, sxy = (T)(sx * sy);
    for (int step = 0; step < ncx + ncy - 1; ++step) {
        const int c = step - r;
        const bool act = row_ok && c >= 0 && c < ncx;
        T psi[4] = {0, 0, 0, 0};
        if (act) {
            const int lx = lx0 + c;
            const int ix = sx > 0 ? lx : a.nx - 1 - lx;
            const int k = iy * a.nx + ix;
            const T sa = a.sig[2 * k], ss = a.sig[2 * k + 1];
            const T sg = sa + ss + a.inv_cdt;
            const T sA = sg * a.area;
            const T* po = a.phi_old + 4 * (size_t)k;
            const double* mm = a.mom + 4 * (size_t)k;
            const T cs = ss * a.area * T(0.07957747154594767);   // sigma_s A / (4 pi)
            const T S0 = cs * po[0] + (T)mm[0] * a.inv_4pi_dt;
            const T S1 = cs * po[1] * T(1.0 / 3.0) + (T)mm[1] * a.inv_4pi_dt;
            const T S2 = cs * po[2] * T(1.0 / 3.0) + (T)mm[2] * a.inv_4pi_dt;
            const T S3 = cs * po[3] * T(1.0 / 9.0) + (T)mm[3] * a.inv_4pi_dt;
            const T by0 = ytr[(q * kSnTile + c) * 2], by1 = ytr[(q * kSnTile + c) * 2 + 1];
            T M[4][4] = {{sA + T(2) * X + T(2) * Y, T(2) * X, T(2) * Y, T(0)},
                         {T(-2) * X, sA / T(3) + T(2) * X + T(2.0 / 3.0) * Y, T(0), T(2.0 / 3.0) * Y},
                         {T(-2) * Y, T(0), sA / T(3) + T(2.0 / 3.0) * X + T(2) * Y, T(2.0 / 3.0) * X},
                         {T(0), T(-2.0 / 3.0) * Y, T(-2.0 / 3.0) * X, sA / T(9) + T(2.0 / 3.0) * (X + Y)}};
            T b[4] = {S0 + T(2) * X * bx0 + T(2) * Y * by0,
                      sxf * S1 - T(2) * X * bx0 + T(2.0 / 3.0) * Y * by1,
                      syf * S2 + T(2.0 / 3.0) * X * bx1 - T(2) * Y * by0,
                      sxy * S3 - T(2.0 / 3.0) * X * bx1 - T(2.0 / 3.0) * Y * by1};
            T ap[4];
            solve4<T>(M, b, ap);
            // outgoing traces in mirrored coordinates
            bx0 = ap[0] + ap[1]; bx1 = ap[2] + ap[3];
            ytr[(q * kSnTile + c) * 2] = ap[0] + ap[2];
            ytr[(q * kSnTile + c) * 2 + 1] = ap[1] + ap[3];
            psi[0] = wq * ap[0]; psi[1] = wq * sxf * ap[1]; psi[2] = wq * syf * ap[2]; psi[3] = wq * sxy * ap[3];
            if (c == ncx - 1) {
                T* d = a.tx + (((size_t)m * a.ny + ly) * a.ntx + tlx) * 2;
                d[0] = bx0; d[1] = bx1;
            }
            if (r == ncy - 1) {
                T* d = a.ty + (((size_t)m * a.nx + (lx0 + c)) * a.nty + tly) * 2;
                d[0] = ap[0] + ap[2]; d[1] = ap[1] + ap[3];
            }
        }
        T* ac = acc + (q * kSnTile + r) * 4;
        ac[0] = psi[0]; ac[1] = psi[1]; ac[2] = psi[2]; ac[3] = psi[3];
        __syncthreads();
        if (q == 0 && act) {
            T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
            for (int qq = 0; qq < a.nq; ++qq) {
                const T* v = acc + (qq * kSnTile + r) * 4;
                s0 += v[0]; s1 += v[1]; s2 += v[2]; s3 += v[3];
            }
            const int lx = lx0 + c;
            const int ix = sx > 0 ? lx : a.nx - 1 - lx;
            T* d = a.phi_quad + ((size_t)quad * a.nx * a.ny + (size_t)iy * a.nx + ix) * 4;
            d[0] = s0; d[1] = s1; d[2] = s2; d[3] = s3;
        }
        __syncthreads();
    }
}

// phi_new = sum of the quadrant partials; norm partials of the change (block order)
template <typename T>
__global__ void sn_reduce_kernel(const T* phi_quad, const T* phi_old, T* phi_new, int ncells, double* part) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double num = 0, den = 0;
    if (k < ncells) {
        const double nrm[4] = {1.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 9.0};
        for (int i = 0; i < 4; ++i) {
            T s = 0;
            for (int qd = 0; qd < 4; ++qd) s += phi_quad[((size_t)qd * ncells + k) * 4 + i];
            phi_new[4 * (size_t)k + i] = s;
            const double d = (double)s - (double)phi_old[4 * (size_t)k + i];
            num += nrm[i] * d * d;
            den += nrm[i] * (double)s * (double)s;
        }
    }
    num = warp_sum(num);
    den = warp_sum(den);
    __shared__ double sn[32], sd[32];
    if ((threadIdx.x & 31) == 0) { sn[threadIdx.x >> 5] = num; sd[threadIdx.x >> 5] = den; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += sn[q]; b += sd[q]; }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void sn_norm_final_kernel(const double* part, int nparts, DevState* st) {
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int i = 0; i < nparts; ++i) { a += part[2 * i]; b += part[2 * i + 1]; }
        st->sn_norm_num = a;
        st->sn_norm_den = b;
    }
}

template <typename T>
__global__ void sn_to_double_kernel(const T* phi, double* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)phi[i];
}

template <typename T>
static cudaError_t sn_iteration_t(hyb_problem* p) {
    cudaStream_t s = p->stream;
    const int nq = p->n_ord / 4;
    SweepArgs<T> a;
    a.nx = p->nx; a.ny = p->ny;
    a.ntx = (p->nx + kSnTile - 1) / kSnTile;
    a.nty = (p->ny + kSnTile - 1) / kSnTile;
    a.nq = nq;
    a.dx = (T)p->dx; a.dy = (T)p->dy; a.area = (T)p->area;
    a.inv_cdt = (T)(1.0 / (p->d.c * p->d.dt));
    a.sig = (const T*)p->sig;
    a.phi_old = (const T*)p->sn_phi_old;
    a.mom = p->mom_d;
    a.inv_4pi_dt = (T)(1.0 / (4.0 * 3.14159265358979323846 * p->d.dt));
    T* qbuf = (T*)p->sn_quadbuf;
    a.qox = qbuf; a.qoy = qbuf + kMaxOrd; a.qw = qbuf + 2 * kMaxOrd;
    a.phi_quad = (T*)p->sn_quad;
    a.tx = (T*)p->sn_tx;
    a.ty = (T*)p->sn_ty;
    const size_t smem = (size_t)nq * kSnTile * (2 + 4) * sizeof(T);
    for (int d = 0; d < a.ntx + a.nty - 1; ++d) {
        a.diag = d;
        const int lo = d - (a.nty - 1) > 0 ? d - (a.nty - 1) : 0;
        const int hi = d < a.ntx - 1 ? d : a.ntx - 1;
        dim3 grid(hi - lo + 1, 4);
        sweep_tile_kernel<T><<<grid, nq * kSnTile, smem, s>>>(a);
    }
    const int g = (p->ncells + 255) / 256;
    sn_reduce_kernel<T><<<g, 256, 0, s>>>((const T*)p->sn_quad, (const T*)p->sn_phi_old, (T*)p->sn_phi, p->ncells,
                                          p->sn_norm);
    sn_norm_final_kernel<<<1, 32, 0, s>>>(p->sn_norm, g, p->st);
    return cudaGetLastError();
}

cudaError_t sn_iteration(hyb_problem* p, int first) {
    if (first) {
        const size_t bytes = (size_t)4 * p->ncells * (p->prec == HYB_FP64 ? 8 : 4);
        cudaError_t e = cudaMemsetAsync(p->sn_phi_old, 0, bytes, p->stream);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = p->prec == HYB_FP64 ? sn_iteration_t<double>(p) : sn_iteration_t<float>(p);
    if (e != cudaSuccess) return e;
    void* t = p->sn_phi; p->sn_phi = p->sn_phi_old; p->sn_phi_old = t;   // newest is now sn_phi_old
    return cudaSuccess;
}

cudaError_t sn_finish(hyb_problem* p) {
    const int n = 4 * p->ncells;
    if (p->prec == HYB_FP64)
        sn_to_double_kernel<double><<<(n + 255) / 256, 256, 0, p->stream>>>((const double*)p->sn_phi_old, p->sn_phi_d, n);
    else
        sn_to_double_kernel<float><<<(n + 255) / 256, 256, 0, p->stream>>>((const float*)p->sn_phi_old, p->sn_phi_d, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_flux(p);
}

}  // namespace hyb
