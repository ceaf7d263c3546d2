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
// registers, so a step needs no block barrier. Strips are pipelined across the warps, so the
// critical path is about (nx + 31) + 32 (ceil(ny/32) - 1) cell solves per sweep. Coordinates are mirrored per quadrant so that every
// sweep runs towards +x,+y; in mirrored coordinates the 4x4 cell system is the same for every
// quadrant and is diagonally dominant, so it is solved by elimination without pivoting. The
// per-ordinate results are summed over ordinates in a fixed order (deterministic).
#include <cuda_runtime.h>

#include <cmath>

#include "hyb_device.cuh"

namespace hyb {

template <typename T>
struct SweepArgs {
    int nx, ny, nq, nord, W;
    T dx, dy;
    const T* sgA;            // (sigma_t + 1/(c dt)) A per cell
    const T* src;            // per cell the four source integrals S_i (un-mirrored)
    const T* qox; const T* qoy; const T* qw;   // ordinates by quadrant: m = quad * nq + q
    T* psi;                  // per ordinate and cell: w_m psi (4 Legendre coefficients)
    int* status;             // device status word (bounded waits)
    const int* conv;         // converged flag: set -> the sweep returns at once
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

template <typename T>
__global__ void sn_source_kernel(int ncells, const T* sig, const T* phi_old, const double* mom, T area,
                                 T inv_4pi_dt, T inv_cdt, T* src, T* sgA) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncells) return;
    const T sa = sig[2 * k], ss = sig[2 * k + 1];
    source4<T>(ss, area, phi_old + 4 * (size_t)k, mom + 4 * (size_t)k, inv_4pi_dt, src + 4 * (size_t)k);
    sgA[k] = (sa + ss + inv_cdt) * area;
}

template <typename T> __device__ __forceinline__ T rcp_(T x) { return T(1) / x; }
template <> __device__ __forceinline__ float rcp_<float>(float x) { return __frcp_rn(x); }

// The mirrored cell system couples {a0, a3} only to {a1, a2}:
//   [ d0  2X  2Y   0 ]        d0 = sA + 2X + 2Y,       d1 = sA/3 + 2X + (2/3)Y,
//   [-2X  d1   0  tY ]        d2 = sA/3 + (2/3)X + 2Y, d3 = sA/9 + (2/3)(X + Y),
//   [-2Y   0  d2  tX ]        tX = (2/3)X, tY = (2/3)Y;
//   [  0 -tY -tX  d3 ]
// eliminating a0 and a3 leaves a symmetric positive 2x2 system for (a1, a2) (Schur complement),
// a short dependency chain: two reciprocals, one 2x2 determinant, back substitution.
template <typename T>
__device__ __forceinline__ void solve_mirrored(T sA, T X, T Y, const T b[4], T ap[4]) {
    const T twoX = T(2) * X, twoY = T(2) * Y, tX = T(2.0 / 3.0) * X, tY = T(2.0 / 3.0) * Y;
    const T d0 = sA + twoX + twoY;
    const T d1 = sA * T(1.0 / 3.0) + twoX + tY;
    const T d2 = sA * T(1.0 / 3.0) + tX + twoY;
    const T d3 = sA * T(1.0 / 9.0) + tX + tY;
    const T i0 = rcp_(d0), i3 = rcp_(d3);
    const T A = d1 + twoX * twoX * i0 + tY * tY * i3;
    const T B = twoX * twoY * i0 + tX * tY * i3;
    const T D = d2 + twoY * twoY * i0 + tX * tX * i3;
    const T r1 = b[1] + twoX * b[0] * i0 - tY * b[3] * i3;
    const T r2 = b[2] + twoY * b[0] * i0 - tX * b[3] * i3;
    const T idet = rcp_(A * D - B * B);
    const T a1 = (D * r1 - B * r2) * idet;
    const T a2 = (A * r2 - B * r1) * idet;
    ap[0] = (b[0] - twoX * a1 - twoY * a2) * i0;
    ap[1] = a1;
    ap[2] = a2;
    ap[3] = (b[3] + tY * a1 + tX * a2) * i3;
}

// Pipelined strip sweep, one CTA per ordinate, W warps. Warp w sweeps strips w, w+W, ... (lane =
// row, one anti-diagonal per step). The trace leaving the top row of strip s goes through a
// shared-memory ring slot (s mod W) to the first row of strip s+1, guarded by produced/consumed
// counters; every wait is bounded and records kStSegments on exhaustion. Dependencies only point
// to lower strips, and all warps of the CTA are resident, so the pipeline always advances.
template <typename T>
__global__ void sweep_pipe_kernel(SweepArgs<T> a) {
    if (*(volatile const int*)a.conv) return;
    extern __shared__ unsigned char smraw[];
    const int W = a.W;
    volatile int* prod = (volatile int*)smraw;
    volatile int* cons = prod + W;
    T* ring = (T*)(smraw + ((2 * W * sizeof(int) + 15) / 16) * 16);   // W x nx x 2
    const int m = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < W) { prod[threadIdx.x] = 0; cons[threadIdx.x] = 0; }
    __syncthreads();
    const int quad = m / a.nq;
    const int sx = (quad == 0 || quad == 3) ? 1 : -1;
    const int sy = (quad <= 1) ? 1 : -1;
    const T sxf = (T)sx, syf = (T)sy, sxy = (T)(sx * sy);
    const T wq = a.qw[m];
    const T X = fabs(a.qox[m]) * a.dy * T(0.5), Y = fabs(a.qoy[m]) * a.dx * T(0.5);
    const T twoX = T(2) * X, twoY = T(2) * Y, tX = T(2.0 / 3.0) * X, tY = T(2.0 / 3.0) * Y;
    T* out = a.psi + (size_t)m * a.nx * a.ny * 4;
    const int nx = a.nx, ny = a.ny;
    const int nstrip = (ny + 31) / 32;
    bool timed_out = false;
    for (int s = warp; s < nstrip; s += W) {
        const int ly = 32 * s + lane;
        const bool row_ok = ly < ny;
        const int iy = sy > 0 ? ly : ny - 1 - ly;
        const int bin = (s - 1 + W) % W, bout = s % W;
        const int qin = ((s - 1) / W) * nx, qout = (s / W) * nx;   // sequence bases of the ring slots
        const bool has_in = s > 0, has_out = s + 1 < nstrip;
        volatile T* rin = ring + (size_t)bin * nx * 2;
        volatile T* rout = ring + (size_t)bout * nx * 2;
        T bx0 = 0, bx1 = 0, oy0 = 0, oy1 = 0;
        int c = -lane;
        // cell data three steps ahead (L2 latency spans several wavefront steps)
        T q0[5] = {0, 0, 0, 0, 1}, q1[5] = {0, 0, 0, 0, 1}, q2[5] = {0, 0, 0, 0, 1};
        auto load = [&](int col, T* d) {
            if (row_ok && col >= 0 && col < nx) {
                const int ix = sx > 0 ? col : nx - 1 - col;
                const size_t k = (size_t)iy * nx + ix;
                const T* sp = a.src + 4 * k;
                d[0] = __ldg(sp); d[1] = __ldg(sp + 1); d[2] = __ldg(sp + 2); d[3] = __ldg(sp + 3);
                d[4] = __ldg(a.sgA + k);
            }
        };
        load(c, q0);
        load(c + 1, q1);
        load(c + 2, q2);
        for (int t = 0; t < nx + 31; ++t, ++c) {
            const T S0 = q0[0], S1 = q0[1], S2 = q0[2], S3 = q0[3], sA = q0[4];
#pragma unroll
            for (int i = 0; i < 5; ++i) { q0[i] = q1[i]; q1[i] = q2[i]; }
            load(c + 3, q2);
            const bool act = row_ok && c >= 0 && c < nx;
            // lane 0 needs the trace of column c from strip s-1; the top lane must not overwrite
            // ring slot column c before strip s+1-W's consumer has read it
            const bool wait_in = has_in && lane == 0 && act;
            const bool wait_out = has_out && lane == 31 && act;
            int spins = 0;
            while (__any_sync(0xffffffffu, (wait_in && prod[bin] < qin + c + 1) ||
                                               (wait_out && cons[bout] < qout + c + 1 - nx))) {
                if (++spins > (1 << 22)) { timed_out = true; break; }
                __nanosleep(32);
            }
            const T u0 = __shfl_up_sync(0xffffffffu, oy0, 1);
            const T u1 = __shfl_up_sync(0xffffffffu, oy1, 1);
            if (act) {
                T by0, by1;
                if (lane == 0) {
                    if (has_in) {
                        by0 = rin[2 * c]; by1 = rin[2 * c + 1];
                        __threadfence_block();
                        cons[bin] = qin + c + 1;
                    } else { by0 = 0; by1 = 0; }
                } else { by0 = u0; by1 = u1; }
                if (c == 0) { bx0 = 0; bx1 = 0; }
                const T b[4] = {S0 + twoX * bx0 + twoY * by0,
                                sxf * S1 - twoX * bx0 + tY * by1,
                                syf * S2 + tX * bx1 - twoY * by0,
                                sxy * S3 - tX * bx1 - tY * by1};
                T ap[4];
                solve_mirrored<T>(sA, X, Y, b, ap);
                bx0 = ap[0] + ap[1]; bx1 = ap[2] + ap[3];
                oy0 = ap[0] + ap[2]; oy1 = ap[1] + ap[3];
                const int ix = sx > 0 ? c : nx - 1 - c;
                T* d = out + ((size_t)iy * nx + ix) * 4;
                d[0] = wq * ap[0]; d[1] = wq * sxf * ap[1]; d[2] = wq * syf * ap[2]; d[3] = wq * sxy * ap[3];
                if (lane == 31 && has_out) {
                    rout[2 * c] = oy0; rout[2 * c + 1] = oy1;
                    __threadfence_block();
                    prod[bout] = qout + c + 1;
                }
            }
            __syncwarp();
            if (timed_out) break;
        }
        if (timed_out) break;
    }
    if (timed_out && lane == 0) atomicOr(a.status, kStSegments);
}

// phi_new = sum over ordinates of w_m psi_m (fixed order); norm partials of the change; the next
// iteration's source integrals from phi_new
template <typename T>
__global__ void sn_reduce_kernel(const T* psi, int nord, const T* phi_old, T* phi_new, int ncells, double* part,
                                 const T* sig, const double* mom, T area, T inv_4pi_dt, T* src, const int* conv) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (*(volatile const int*)conv) {
        // converged earlier: carry the solution forward so the buffer alternation stays aligned
        if (k < ncells)
            for (int i = 0; i < 4; ++i) phi_new[4 * (size_t)k + i] = phi_old[4 * (size_t)k + i];
        return;
    }
    double num = 0, den = 0;
    if (k < ncells) {
        const double nrm[4] = {1.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 9.0};
        T s[4] = {0, 0, 0, 0};
        for (int m = 0; m < nord; ++m) {
            const T* v = psi + ((size_t)m * ncells + k) * 4;
            s[0] += v[0]; s[1] += v[1]; s[2] += v[2]; s[3] += v[3];
        }
        for (int i = 0; i < 4; ++i) {
            phi_new[4 * (size_t)k + i] = s[i];
            const double d = (double)s[i] - (double)phi_old[4 * (size_t)k + i];
            num += nrm[i] * d * d;
            den += nrm[i] * (double)s[i] * (double)s[i];
        }
        source4<T>(sig[2 * k + 1], area, s, mom + 4 * (size_t)k, inv_4pi_dt, src + 4 * (size_t)k);
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

// SI stop test on the device: ||phi_new - phi_old|| <= tol ||phi_new|| (or no source at all)
__global__ void sn_norm_final_kernel(const double* part, int nparts, DevState* st, double tol) {
    if (*(volatile int*)&st->sn_conv) return;
    double a = 0, b = 0;
    for (int i = threadIdx.x; i < nparts; i += 32) { a += part[2 * i]; b += part[2 * i + 1]; }
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x == 0) {
        st->sn_norm_num = a;
        st->sn_norm_den = b;
        st->sn_iters += 1;
        if (b == 0.0 || sqrt(a) <= tol * sqrt(b)) st->sn_conv = 1;
    }
}

// start of a solve: clear the stop state; the iterate starts from the previous solution
// (warm start, re-read from its FP64 copy) or from zero
template <typename T>
__global__ void sn_seed_kernel(const double* prev, T* phi, int n, const DevState* st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) phi[i] = st->sn_warm ? (T)prev[i] : T(0);
}

__global__ void sn_done_kernel(DevState* st, int warm) { st->sn_warm = warm; }

template <typename T>
__global__ void sn_to_double_kernel(const T* phi, double* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)phi[i];
}

template <typename T>
static int sweep_warps(const hyb_problem* p, size_t* smem) {
    const int nstrip = (p->ny + 31) / 32;
    const size_t per = (size_t)p->nx * 2 * sizeof(T);
    int W = nstrip < 16 ? nstrip : 16;
    while (W > 1 && (size_t)W * per + 256 > 160 * 1024) --W;
    *smem = ((2 * W * sizeof(int) + 15) / 16) * 16 + (size_t)W * per;
    return W;
}

template <typename T>
static cudaError_t sn_iteration_t(hyb_problem* p, int first) {
    cudaStream_t s = p->stream;
    const int g = (p->ncells + 255) / 256;
    T* src = (T*)p->sn_quad;                      // 4 per cell
    T* sgA = src + 4 * (size_t)p->ncells;         // 1 per cell
    const T inv4pidt = (T)(1.0 / (4.0 * 3.14159265358979323846 * p->d.dt));
    if (first)
        sn_source_kernel<T><<<g, 256, 0, s>>>(p->ncells, (const T*)p->sig, (const T*)p->sn_phi_old, p->mom_d,
                                              (T)p->area, inv4pidt, (T)(1.0 / (p->d.c * p->d.dt)), src, sgA);
    SweepArgs<T> a;
    a.nx = p->nx; a.ny = p->ny;
    a.nq = p->n_ord / 4;
    a.nord = p->n_ord;
    a.dx = (T)p->dx; a.dy = (T)p->dy;
    a.sgA = sgA;
    a.src = src;
    T* qbuf = (T*)p->sn_quadbuf;
    a.qox = qbuf; a.qoy = qbuf + kMaxOrd; a.qw = qbuf + 2 * kMaxOrd;
    a.psi = (T*)p->sn_psi;
    a.status = &p->st->status;
    a.conv = &p->st->sn_conv;
    size_t smem = 0;
    a.W = sweep_warps<T>(p, &smem);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(sweep_pipe_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    sweep_pipe_kernel<T><<<p->n_ord, 32 * a.W, smem, s>>>(a);
    sn_reduce_kernel<T><<<g, 256, 0, s>>>((const T*)p->sn_psi, p->n_ord, (const T*)p->sn_phi_old, (T*)p->sn_phi,
                                          p->ncells, p->sn_norm, (const T*)p->sig, p->mom_d, (T)p->area, inv4pidt,
                                          src, &p->st->sn_conv);
    sn_norm_final_kernel<<<1, 32, 0, s>>>(p->sn_norm, g, p->st, sn_tol_eff(p));
    return cudaGetLastError();
}

cudaError_t sn_start(hyb_problem* p) {
    cudaError_t e = cudaMemsetAsync(&p->st->sn_conv, 0, 2 * sizeof(int), p->stream);
    if (e != cudaSuccess) return e;
    const int n = 4 * p->ncells, g = (n + 255) / 256;
    if (p->prec == HYB_FP64)
        sn_seed_kernel<double><<<g, 256, 0, p->stream>>>(p->sn_phi_d, (double*)p->sn_phi_old, n, p->st);
    else
        sn_seed_kernel<float><<<g, 256, 0, p->stream>>>(p->sn_phi_d, (float*)p->sn_phi_old, n, p->st);
    return cudaGetLastError();
}

cudaError_t sn_iteration(hyb_problem* p, int first) {
    cudaError_t e = p->prec == HYB_FP64 ? sn_iteration_t<double>(p, first) : sn_iteration_t<float>(p, first);
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
    sn_done_kernel<<<1, 1, 0, p->stream>>>(p->st, p->d.sn_warm_start ? 1 : 0);
    return launch_flux(p);
}

}  // namespace hyb
