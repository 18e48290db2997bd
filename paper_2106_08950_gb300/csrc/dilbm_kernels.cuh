// Device code of the DI-LBM step on sm_103a.
//
// One time step (the paper's procedure, Sec. 2.3) is three kernels:
//   sweep_kernel      -- every node: pull-stream, edge extrapolation, solid
//                        fraction (Eq. 14), corrected velocity (Eq. 17),
//                        collision with the force term (Eqs. 13, 15), and the
//                        node's share of force/torque (Eqs. 18-19) summed per
//                        tile and per nearby particle into FP64 partials;
//   reduce_kernel     -- per particle: fixed-order FP64 sum of its partials
//                        and the Wan-Turek repulsion (Eqs. 28-29);
//   integrate_bin_kernel -- per particle: Newton-Euler update (Eqs. 22-24),
//                        then binning of the particle into the lattice tiles
//                        its phi tail reaches, for the next sweep.
//
// Populations are stored as deviations d_i = f_i - w_i (structure of arrays:
// 9 planes of ny rows of `pitch` elements), in FP32, FP16 or BF16; all
// arithmetic is FP32, force/torque accumulation and particle state FP64.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dilbm {

constexpr int TILE_W = 128;   // nodes per tile row: 32 lanes x 4 nodes
constexpr int TILE_H = 8;     // rows per tile: one warp per row
constexpr int VEC = 4;        // nodes per thread
constexpr int MAXC = 32;      // candidate particles per tile
constexpr float PHI_CUT_WIDTHS = 6.0f;   // phi tail kept up to 6 interface widths

enum : int { SIDE_PERIODIC = 0, SIDE_VELOCITY = 1, SIDE_PRESSURE = 2 };
enum : int { WEST = 0, EAST = 1, SOUTH = 2, NORTH = 3 };
enum : int { ERR_UNSTABLE = 1, ERR_OVERFLOW = 2 };

// D2Q9 directions of Eq. 3 and weights of Eq. 4.
__host__ __device__ constexpr int cxof(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int cyof(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr float wof(int i) { return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f); }

// ------------------------------------------------------------ storage types
template <typename T> struct Storage;

template <> struct Storage<float> {
    static __device__ __forceinline__ float4 load4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
    static __device__ __forceinline__ float load1(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ void store4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
    static __device__ __forceinline__ void store1(float *p, float v) { *p = v; }
    static __host__ __device__ float from_float(float v) { return v; }
};

template <> struct Storage<__half> {
    static __device__ __forceinline__ float4 load4(const __half *p) {
        uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
        __half2 a = *reinterpret_cast<__half2 *>(&u.x), b = *reinterpret_cast<__half2 *>(&u.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    static __device__ __forceinline__ float load1(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void store4(__half *p, float4 v) {
        __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t *>(&a);
        u.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = u;
    }
    static __device__ __forceinline__ void store1(__half *p, float v) { *p = __float2half_rn(v); }
};

template <> struct Storage<__nv_bfloat16> {
    static __device__ __forceinline__ float4 load4(const __nv_bfloat16 *p) {
        uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
        __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&u.x), b = *reinterpret_cast<__nv_bfloat162 *>(&u.y);
        float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    static __device__ __forceinline__ float load1(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void store4(__nv_bfloat16 *p, float4 v) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t *>(&a);
        u.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = u;
    }
    static __device__ __forceinline__ void store1(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// ------------------------------------------------------------ parameters
struct Particles {      // structure of arrays, device memory
    double *x, *y, *r, *ux, *uy, *omega, *theta, *rho_s;
    float *xf, *yf;     // FP32 copy of the centre, for cheap proximity tests
    int *fixed;
};

struct Lattice {
    int nx, ny, pitch;          // nodes; row pitch in elements (multiple of 4)
    long long plane;            // elements per population plane (ny * pitch)
    int ntx, nty;               // tiles along x and y
    int per_x, per_y;           // periodic axes
    int side_kind[4];
    float side_ux[4], side_uy[4], side_drho[4];   // drho = rho_b - 1
};

struct Physics {
    float omega;                // 1 / tau
    float kf;                   // 1 - 1/(2 tau): prefactor of F_i (Eq. 15)
    float kforce;               // kf (Eq. 18 as printed) or 1 (momentum exchange)
    float four_over_eps;        // 4 / epsilon: phi = 1 / (1 + exp(-4 l / eps))
    float cut;                  // phi tail kept while l >= -cut
    double cut_d;
};

struct Bins {
    int *count;                 // per tile: particles binned (may exceed MAXC)
    int *ids;                   // per tile: MAXC particle ids
    double *partial;            // per tile and slot: Fx, Fy, T
};

// ------------------------------------------------------------ small helpers
__device__ __forceinline__ int wrap_or_clamp(int v, int n, int periodic) {
    if (periodic) return v < 0 ? v + n : (v >= n ? v - n : v);
    return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

// Equilibrium deviation f^eq_i(rho, u) - w_i (Eq. 2) with rho = 1 + drho.
__device__ __forceinline__ float eq_dev(int i, float drho, float rho, float ux, float uy, float usq) {
    const float cu = cxof(i) * ux + cyof(i) * uy;
    return wof(i) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
}

// Tile ranges along one axis covered by [X - R, X + R] (a disc's bounding
// interval); periodic intervals wrap and may split in two.  Shared by the
// binning and the reduction so both visit the same tiles in the same order.
struct AxisTiles {
    int n;
    int lo[2], hi[2];
};

__host__ __device__ inline AxisTiles axis_tiles(double X, double R, int n, int tile, int ntiles, int periodic) {
    AxisTiles t;
    int il = (int)floor(X - R), ih = (int)ceil(X + R);
    if (periodic) {
        if (ih - il + 1 >= n) { t.n = 1; t.lo[0] = 0; t.hi[0] = ntiles - 1; return t; }
        int a = ((il % n) + n) % n, b = ((ih % n) + n) % n;
        if (a <= b) { t.n = 1; t.lo[0] = a / tile; t.hi[0] = b / tile; return t; }
        int first_hi = b / tile, second_lo = a / tile;
        if (first_hi >= second_lo) { t.n = 1; t.lo[0] = 0; t.hi[0] = ntiles - 1; return t; }
        t.n = 2; t.lo[0] = 0; t.hi[0] = first_hi; t.lo[1] = second_lo; t.hi[1] = ntiles - 1;
        return t;
    }
    il = il < 0 ? 0 : il;
    ih = ih > n - 1 ? n - 1 : ih;
    if (il > ih) { t.n = 0; return t; }
    t.n = 1; t.lo[0] = il / tile; t.hi[0] = ih / tile;
    return t;
}

// ------------------------------------------------------------ the sweep
// Mode: STEP writes the collided populations and the force partials; FIELDS
// writes rho, the corrected velocity and phi of the streamed state instead.
enum : int { MODE_STEP = 0, MODE_FIELDS = 1 };

struct FieldsOut {
    float *rho, *ux, *uy, *phi;   // dense [ny][nx]
};

template <typename T>
__device__ __forceinline__ void pull_node_scalar(const T *__restrict__ src, const Lattice &L, int x, int y, float d[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sx = wrap_or_clamp(x - cxof(i), L.nx, L.per_x);
        int sy = wrap_or_clamp(y - cyof(i), L.ny, L.per_y);
        d[i] = Storage<T>::load1(src + i * L.plane + (long long)sy * L.pitch + sx);
    }
}

// Non-equilibrium extrapolation at an edge node (x, y) (Guo et al. 2002, as
// the paper's Sec. 3 uses): d_b = deq(rho_b, u_b) + d_n - deq(rho_n, u_n),
// with n the inner neighbour (diagonal at corners; corners take the
// south/north condition).
template <typename T>
__device__ __forceinline__ void edge_extrapolate(const T *__restrict__ src, const Lattice &L, int x, int y, float d[9]) {
    const int onx = !L.per_x && (x == 0 || x == L.nx - 1);
    const int ony = !L.per_y && (y == 0 || y == L.ny - 1);
    const int side = ony ? (y == 0 ? SOUTH : NORTH) : (x == 0 ? WEST : EAST);
    const int xn = onx ? (x == 0 ? 1 : L.nx - 2) : x;
    const int yn = ony ? (y == 0 ? 1 : L.ny - 2) : y;
    float dn[9];
    pull_node_scalar<T>(src, L, xn, yn, dn);
    float drn = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        drn += dn[i];
        jx += cxof(i) * dn[i];
        jy += cyof(i) * dn[i];
    }
    const float rhon = 1.0f + drn;
    const float unx = jx / rhon, uny = jy / rhon;
    // select the side's parameters without indexing the kernel-parameter arrays
    int kind = L.side_kind[0];
    float sux = L.side_ux[0], suy = L.side_uy[0], sdr = L.side_drho[0];
#pragma unroll
    for (int k = 1; k < 4; ++k)
        if (side == k) { kind = L.side_kind[k]; sux = L.side_ux[k]; suy = L.side_uy[k]; sdr = L.side_drho[k]; }
    float drb, ubx, uby;
    if (kind == SIDE_VELOCITY) {
        drb = drn; ubx = sux; uby = suy;
    } else {
        drb = sdr; ubx = unx; uby = uny;
    }
    const float rhob = 1.0f + drb;
    const float usqb = ubx * ubx + uby * uby, usqn = unx * unx + uny * uny;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        d[i] = eq_dev(i, drb, rhob, ubx, uby, usqb) + (dn[i] - eq_dev(i, drn, rhon, unx, uny, usqn));
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256)
sweep_kernel(const T *__restrict__ src, T *__restrict__ dst, Lattice L, Physics ph,
             Particles P, Bins B, FieldsOut fo, int *__restrict__ err)
{
    __shared__ int s_n;
    __shared__ int s_id[MAXC];
    __shared__ float s_cxh[MAXC], s_cxl[MAXC], s_cyh[MAXC], s_cyl[MAXC];
    __shared__ float s_r[MAXC], s_ux[MAXC], s_uy[MAXC], s_om[MAXC];
    __shared__ float s_red[TILE_H][MAXC][3];

    const int lane = threadIdx.x, wy = threadIdx.y;
    const int tx = blockIdx.x, ty = blockIdx.y;
    const int tile = ty * L.ntx + tx;
    const int tx0 = tx * TILE_W, ty0 = ty * TILE_H;
    const int tid = wy * 32 + lane;

    // Candidate particles of this tile: centre relative to the tile origin,
    // minimum image about the tile centre, as an FP32 hi + lo pair.
    if (tid == 0) {
        int n = B.count ? B.count[tile] : 0;
        s_n = n > MAXC ? MAXC : n;
    }
    __syncthreads();
    const int ncand = s_n;
    if (tid < ncand) {
        const int q = B.ids[tile * MAXC + tid];
        double cx = P.x[q] - (double)tx0, cy = P.y[q] - (double)ty0;
        if (L.per_x) {
            const double h = 0.5 * TILE_W;
            while (cx - h >= 0.5 * L.nx) cx -= L.nx;
            while (cx - h < -0.5 * L.nx) cx += L.nx;
        }
        if (L.per_y) {
            const double h = 0.5 * TILE_H;
            while (cy - h >= 0.5 * L.ny) cy -= L.ny;
            while (cy - h < -0.5 * L.ny) cy += L.ny;
        }
        const float cxh = (float)cx, cyh = (float)cy;
        s_id[tid] = q;
        s_cxh[tid] = cxh; s_cxl[tid] = (float)(cx - (double)cxh);
        s_cyh[tid] = cyh; s_cyl[tid] = (float)(cy - (double)cyh);
        s_r[tid] = (float)P.r[q];
        s_ux[tid] = (float)P.ux[q];
        s_uy[tid] = (float)P.uy[q];
        s_om[tid] = (float)P.omega[q];
    }
    __syncthreads();

    const int y = ty0 + wy;
    const int x0 = tx0 + lane * VEC;
    const bool row_ok = y < L.ny;
    const int yc = row_ok ? y : L.ny - 1;               // rows past the end read a valid row
    const int xl = x0 <= L.pitch - VEC ? x0 : L.pitch - VEC;

    // ---- pull-stream: f_i(x, t+1) = f'_i(x - c_i, t), 4 nodes per thread
    float d[9][VEC];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = cxof(i), cy = cyof(i);
        const int sy = wrap_or_clamp(yc - cy, L.ny, L.per_y);
        const T *row = src + i * L.plane + (long long)sy * L.pitch;
        const float4 v = Storage<T>::load4(row + xl);
        if (cx == 0) {
            d[i][0] = v.x; d[i][1] = v.y; d[i][2] = v.z; d[i][3] = v.w;
        } else if (cx == 1) {
            float left = __shfl_up_sync(0xffffffffu, v.w, 1);
            if (lane == 0) left = Storage<T>::load1(row + wrap_or_clamp(x0 - 1, L.nx, L.per_x));
            d[i][0] = left; d[i][1] = v.x; d[i][2] = v.y; d[i][3] = v.z;
        } else {
            float right = __shfl_down_sync(0xffffffffu, v.x, 1);
            if (lane == 31 || x0 + VEC >= L.nx) {
                // lanes past the row end may sit more than one period beyond it
                const int xr = x0 + VEC;
                right = Storage<T>::load1(row + (L.per_x ? xr % L.nx : (xr < L.nx ? xr : L.nx - 1)));
            }
            d[i][0] = v.y; d[i][1] = v.z; d[i][2] = v.w; d[i][3] = right;
            // the row's last node when nx is not a multiple of 4: its right
            // neighbour wraps to column 0, not the padding in this vector
            const int kl = L.nx - 1 - x0;
            if (kl >= 0 && kl < VEC - 1) {
                const float wv = Storage<T>::load1(row + wrap_or_clamp(L.nx, L.nx, L.per_x));
#pragma unroll
                for (int k = 0; k < VEC - 1; ++k)
                    if (k == kl) d[i][k] = wv;
            }
        }
    }

    const bool edge_tile = (!L.per_x && (tx0 == 0 || tx0 + TILE_W >= L.nx)) ||
                           (!L.per_y && (ty0 == 0 || ty0 + TILE_H >= L.ny));

    float acc[VEC][3];     // per-node force / torque contribution
    int own[VEC];          // owning slot per node, -1 if none
    bool bad = false;

#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        const int x = x0 + k;
        const bool active = row_ok && x < L.nx;
        own[k] = -1;
        acc[k][0] = acc[k][1] = acc[k][2] = 0.f;
        float dk[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) dk[i] = d[i][k];
        if (edge_tile && active) {
            const bool onx = !L.per_x && (x == 0 || x == L.nx - 1);
            const bool ony = !L.per_y && (y == 0 || y == L.ny - 1);
            if (onx || ony) edge_extrapolate<T>(src, L, x, y, dk);
        }

        // ---- moments (Eq. 5, Eq. 16)
        const float drho = ((dk[0] + dk[1]) + (dk[2] + dk[3])) + ((dk[4] + dk[5]) + (dk[6] + dk[7])) + dk[8];
        const float rho = 1.0f + drho;
        const float jx = (dk[1] - dk[3]) + (dk[5] - dk[6]) + (dk[8] - dk[7]);
        const float jy = (dk[2] - dk[4]) + (dk[5] + dk[6]) - (dk[7] + dk[8]);
        const float uax = jx / rho, uay = jy / rho;

        // ---- solid fraction (Eq. 14) from the tile's candidates: max rule
        float phi = 0.f, usx = 0.f, usy = 0.f, rx = 0.f, ry = 0.f;
        int best = -1, best_id = 0x7fffffff;
        for (int c = 0; c < ncand; ++c) {
            float dx = ((float)(x - tx0) - s_cxh[c]) - s_cxl[c];
            float dy = ((float)(y - ty0) - s_cyh[c]) - s_cyl[c];
            if (L.per_x) { if (dx >= 0.5f * L.nx) dx -= L.nx; else if (dx < -0.5f * L.nx) dx += L.nx; }
            if (L.per_y) { if (dy >= 0.5f * L.ny) dy -= L.ny; else if (dy < -0.5f * L.ny) dy += L.ny; }
            const float rr = s_r[c] + ph.cut;
            const float d2 = dx * dx + dy * dy;
            if (d2 > rr * rr) continue;
            const float l = s_r[c] - sqrtf(d2);
            if (l < -ph.cut) continue;
            // (1 + tanh(2l/eps)) / 2 == 1 / (1 + exp(-4l/eps))
            const float pc = 1.0f / (1.0f + expf(-ph.four_over_eps * l));
            const int id = s_id[c];
            if (pc > phi || (pc == phi && pc > 0.f && id < best_id)) {
                phi = pc; best = c; best_id = id; rx = dx; ry = dy;
            }
        }
        if (best >= 0) {
            usx = s_ux[best] - s_om[best] * ry;   // u_s = U + omega x r
            usy = s_uy[best] + s_om[best] * rx;
        }

        // ---- corrected velocity (Eq. 17)
        const float hx = 0.5f * phi * (usx - uax), hy = 0.5f * phi * (usy - uay);
        const float ux = uax + hx, uy = uay + hy;

        if (MODE == MODE_FIELDS) {
            if (active) {
                const long long o = (long long)y * L.nx + x;
                if (fo.rho) fo.rho[o] = rho;
                if (fo.ux) fo.ux[o] = ux;
                if (fo.uy) fo.uy[o] = uy;
                if (fo.phi) fo.phi[o] = phi;
            }
            continue;
        }

        if (active && (!(rho > 0.0f) || !isfinite(uax + uay))) bad = true;

        // ---- collision with the force term (Eqs. 2, 13, 15)
        const float usq = ux * ux + uy * uy;
        if (best >= 0) {
            const float dux = usx - uax, duy = usy - uay;
            const float ssq = (usx * usx + usy * usy) - (uax * uax + uay * uay);
            const float kr = ph.kf * rho * phi;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float cx = (float)cxof(i), cy = (float)cyof(i);
                const float cus = cx * usx + cy * usy, cua = cx * uax + cy * uay;
                const float Fi = wof(i) * (3.0f * (cx * dux + cy * duy) + 4.5f * (cus * cus - cua * cua) - 1.5f * ssq);
                const float deq = eq_dev(i, drho, rho, ux, uy, usq);
                dk[i] = dk[i] - ph.omega * (dk[i] - deq) + kr * Fi;
            }
            // Eqs. 18-19 per node, by the closed form sum_i F_i c_i = kf rho (u_s - u*)
            if (active) {
                const float s = -phi * ph.kforce * rho;
                const float gx = s * dux, gy = s * duy;
                own[k] = best;
                acc[k][0] = gx; acc[k][1] = gy; acc[k][2] = rx * gy - ry * gx;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float deq = eq_dev(i, drho, rho, ux, uy, usq);
                dk[i] = dk[i] - ph.omega * (dk[i] - deq);
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i][k] = dk[i];
    }

    if (MODE == MODE_FIELDS) return;

    if (bad) atomicOr(err, ERR_UNSTABLE);

    // ---- store the collided populations
    if (row_ok) {
        const bool full = x0 + VEC <= L.nx;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            T *row = dst + i * L.plane + (long long)y * L.pitch;
            if (full) {
                Storage<T>::store4(row + x0, make_float4(d[i][0], d[i][1], d[i][2], d[i][3]));
            } else {
#pragma unroll
                for (int k = 0; k < VEC; ++k)
                    if (x0 + k < L.nx) Storage<T>::store1(row + x0 + k, d[i][k]);
            }
        }
    }

    // ---- per-tile, per-candidate force / torque partials (FP64 across warps)
    if (ncand == 0) return;
    for (int c = 0; c < ncand; ++c) {
        float v0 = 0.f, v1 = 0.f, v2 = 0.f;
#pragma unroll
        for (int k = 0; k < VEC; ++k)
            if (own[k] == c) { v0 += acc[k][0]; v1 += acc[k][1]; v2 += acc[k][2]; }
        if (__any_sync(0xffffffffu, v0 != 0.f || v1 != 0.f || v2 != 0.f)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                v2 += __shfl_xor_sync(0xffffffffu, v2, o);
            }
        }
        if (lane == 0) { s_red[wy][c][0] = v0; s_red[wy][c][1] = v1; s_red[wy][c][2] = v2; }
    }
    __syncthreads();
    if (tid < ncand * 3) {
        const int c = tid / 3, comp = tid % 3;
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < TILE_H; ++w) s += (double)s_red[w][c][comp];
        B.partial[((long long)tile * MAXC + c) * 3 + comp] = s;
    }
}

// ------------------------------------------------------------ particles
struct BodyParams {
    int np;
    double gx, gy, rho_f;
    double eps_p, eps_p2, eps_w, eps_w2, xi;
};

// One warp per particle: fixed-order FP64 sum of the particle's tile partials
// (Eqs. 18-19), then the Wan-Turek force (Eqs. 28-29) from the other
// particles (lanes stride over them) and from the walls.
__global__ void reduce_kernel(Lattice L, Physics ph, Particles P, Bins B, BodyParams bp,
                              double *__restrict__ force, double *__restrict__ fcol)
{
    const int lane = threadIdx.x & 31;
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= bp.np) return;
    const double X = P.x[p], Y = P.y[p], r = P.r[p];

    if (lane == 0) {
        const double R = r + ph.cut_d;
        const AxisTiles ax = axis_tiles(X, R, L.nx, TILE_W, L.ntx, L.per_x);
        const AxisTiles ay = axis_tiles(Y, R, L.ny, TILE_H, L.nty, L.per_y);
        double fx = 0.0, fy = 0.0, tq = 0.0;
        for (int a = 0; a < ay.n; ++a)
            for (int ty = ay.lo[a]; ty <= ay.hi[a]; ++ty)
                for (int b = 0; b < ax.n; ++b)
                    for (int tx = ax.lo[b]; tx <= ax.hi[b]; ++tx) {
                        const int t = ty * L.ntx + tx;
                        int n = B.count[t];
                        n = n > MAXC ? MAXC : n;
                        for (int s = 0; s < n; ++s)
                            if (B.ids[t * MAXC + s] == p) {
                                const double *q = B.partial + ((long long)t * MAXC + s) * 3;
                                fx += q[0]; fy += q[1]; tq += q[2];
                                break;
                            }
                    }
        force[3 * p] = fx; force[3 * p + 1] = fy; force[3 * p + 2] = tq;
    }

    // particle-particle repulsion
    double cx = 0.0, cy = 0.0;
    const float xf = P.xf[p], yf = P.yf[p], rf = (float)r;
    for (int j = lane; j < bp.np; j += 32) {
        if (j == p) continue;
        float dxf = xf - P.xf[j], dyf = yf - P.yf[j];
        if (L.per_x) { if (dxf >= 0.5f * L.nx) dxf -= L.nx; else if (dxf < -0.5f * L.nx) dxf += L.nx; }
        if (L.per_y) { if (dyf >= 0.5f * L.ny) dyf -= L.ny; else if (dyf < -0.5f * L.ny) dyf += L.ny; }
        const float lim = rf + (float)P.r[j] + (float)bp.xi + 0.05f;
        if (dxf * dxf + dyf * dyf > lim * lim) continue;
        double dx = X - P.x[j], dy = Y - P.y[j];
        if (L.per_x) { while (dx >= 0.5 * L.nx) dx -= L.nx; while (dx < -0.5 * L.nx) dx += L.nx; }
        if (L.per_y) { while (dy >= 0.5 * L.ny) dy -= L.ny; while (dy < -0.5 * L.ny) dy += L.ny; }
        const double d = sqrt(dx * dx + dy * dy), rr = r + P.r[j];
        double s = 0.0;
        if (d <= rr) s = (rr - d) / bp.eps_p2;
        else if (d <= rr + bp.xi) s = (rr + bp.xi - d) * (rr + bp.xi - d) / bp.eps_p;
        cx += s * dx;
        cy += s * dy;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cx += __shfl_xor_sync(0xffffffffu, cx, o);
        cy += __shfl_xor_sync(0xffffffffu, cy, o);
    }
    if (lane == 0) {
        // wall repulsion: mirror image across each non-periodic wall
        for (int w = 0; w < 4; ++w) {
            if (L.side_kind[w] == SIDE_PERIODIC) continue;
            double ix = X, iy = Y;
            if (w == WEST) ix = -X;
            if (w == EAST) ix = 2.0 * (L.nx - 1) - X;
            if (w == SOUTH) iy = -Y;
            if (w == NORTH) iy = 2.0 * (L.ny - 1) - Y;
            const double dx = X - ix, dy = Y - iy;
            const double d = sqrt(dx * dx + dy * dy), rr = 2.0 * r;
            double s = 0.0;
            if (d <= rr) s = (rr - d) / bp.eps_w2;
            else if (d <= rr + bp.xi) s = (rr + bp.xi - d) * (rr + bp.xi - d) / bp.eps_w;
            cx += s * dx;
            cy += s * dy;
        }
        fcol[2 * p] = cx;
        fcol[2 * p + 1] = cy;
    }
}

// One thread per particle: symplectic Euler of Eqs. 22-24 (dt = 1), then
// binning of the particle into every tile its phi tail reaches.
__global__ void integrate_bin_kernel(Lattice L, Physics ph, Particles P, Bins B, BodyParams bp,
                                     const double *__restrict__ force, const double *__restrict__ fcol,
                                     int integrate, int *__restrict__ err)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= bp.np) return;
    double X = P.x[p], Y = P.y[p];
    const double r = P.r[p];
    if (integrate && !P.fixed[p]) {
        const double m = P.rho_s[p] * 3.14159265358979323846 * r * r;
        const double I = 0.5 * m * r * r;
        const double wgt = (1.0 - bp.rho_f / P.rho_s[p]) * m;   // buoyancy-reduced weight / g
        double ux = P.ux[p] + (force[3 * p] + fcol[2 * p] + wgt * bp.gx) / m;
        double uy = P.uy[p] + (force[3 * p + 1] + fcol[2 * p + 1] + wgt * bp.gy) / m;
        double om = P.omega[p] + force[3 * p + 2] / I;
        X += ux;
        Y += uy;
        if (L.per_x) { X = fmod(X, (double)L.nx); if (X < 0.0) X += L.nx; }
        if (L.per_y) { Y = fmod(Y, (double)L.ny); if (Y < 0.0) Y += L.ny; }
        P.ux[p] = ux; P.uy[p] = uy; P.omega[p] = om;
        P.theta[p] += om;
        P.x[p] = X; P.y[p] = Y;
    }
    P.xf[p] = (float)X;
    P.yf[p] = (float)Y;
    const double R = r + ph.cut_d;
    const AxisTiles ax = axis_tiles(X, R, L.nx, TILE_W, L.ntx, L.per_x);
    const AxisTiles ay = axis_tiles(Y, R, L.ny, TILE_H, L.nty, L.per_y);
    for (int a = 0; a < ay.n; ++a)
        for (int ty = ay.lo[a]; ty <= ay.hi[a]; ++ty)
            for (int b = 0; b < ax.n; ++b)
                for (int tx = ax.lo[b]; tx <= ax.hi[b]; ++tx) {
                    const int t = ty * L.ntx + tx;
                    const int s = atomicAdd(&B.count[t], 1);
                    if (s < MAXC) B.ids[t * MAXC + s] = p;
                    else atomicOr(err, ERR_OVERFLOW);
                }
}

// ------------------------------------------------------------ conversions
// Populations <-> FP64 f_i (dense 9 x ny x nx) for checkpoints.
template <typename T>
__global__ void export_kernel(const T *__restrict__ src, Lattice L, double *__restrict__ out) {
    const long long n = (long long)L.nx * L.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 9 * n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / n);
        const long long r = k - i * n;
        const int y = (int)(r / L.nx), x = (int)(r - (long long)y * L.nx);
        out[k] = (double)Storage<T>::load1(src + i * L.plane + (long long)y * L.pitch + x) + (double)wof(i);
    }
}

template <typename T>
__global__ void import_kernel(T *__restrict__ dst, Lattice L, const double *__restrict__ in) {
    const long long n = (long long)L.nx * L.ny;
    // the same FP32 weights the deviations are taken against, so that an
    // exported state imports back bit for bit
    const double w[9] = {wof(0), wof(1), wof(2), wof(3), wof(4), wof(5), wof(6), wof(7), wof(8)};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 9 * n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / n);
        const long long r = k - i * n;
        const int y = (int)(r / L.nx), x = (int)(r - (long long)y * L.nx);
        Storage<T>::store1(dst + i * L.plane + (long long)y * L.pitch + x, (float)(in[k] - w[i]));
    }
}

// Uniform initial state f^eq(rho0, u0) written as deviations on every node.
template <typename T>
__global__ void init_kernel(T *__restrict__ dst, Lattice L, float drho, float ux, float uy) {
    const long long n = (long long)L.nx * L.ny;
    const float rho = 1.0f + drho, usq = ux * ux + uy * uy;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 9 * n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / n);
        const long long r = k - i * n;
        const int y = (int)(r / L.nx), x = (int)(r - (long long)y * L.nx);
        float v = 0.f;
        switch (i) {
#define DILBM_CASE(I) case I: v = eq_dev(I, drho, rho, ux, uy, usq); break;
            DILBM_CASE(0) DILBM_CASE(1) DILBM_CASE(2) DILBM_CASE(3) DILBM_CASE(4)
            DILBM_CASE(5) DILBM_CASE(6) DILBM_CASE(7) DILBM_CASE(8)
#undef DILBM_CASE
        }
        Storage<T>::store1(dst + i * L.plane + (long long)y * L.pitch + x, v);
    }
}

}  // namespace dilbm
