// Device code of the DI-LBM step on sm_103a.
//
// One time step (the paper's procedure, Sec. 2.3) is two kernels:
//   sweep_kernel     -- every node: pull-stream, edge extrapolation, solid
//                       fraction (Eq. 14), corrected velocity (Eq. 17),
//                       collision with the force term (Eqs. 13, 15), and the
//                       node's share of force/torque (Eqs. 18-19) summed per
//                       row segment and nearby particle;
//   particles_kernel -- one warp per particle: fixed-order FP64 sum of its
//                       partials (Eqs. 18-19), Wan-Turek repulsion (Eqs.
//                       28-29), Newton-Euler update (Eqs. 22-24), then binning
//                       of the particle into the lattice tiles its phi tail
//                       reaches, for the next sweep.
//
// Populations are stored as deviations d_i = f_i - w_i (structure of arrays:
// 9 planes of ny rows of `pitch` elements), in FP32, FP16 or BF16; arithmetic
// is FP32, force/torque accumulation and particle state FP64.  Particle
// positions and the tile bins are double-buffered by step parity, so a step
// reads one copy and writes the other.
//
// The sweep is a persistent kernel: each warp walks row segments of 128 nodes
// and streams every segment's nine source rows (plus a 16-byte halo on each
// side) into shared memory with bulk asynchronous copies (cp.async.bulk,
// completion on an mbarrier); once a segment's rows have been read, the copy
// of the warp's next segment is issued into the same buffer, so it is in
// flight while the current segment is collided.  Each lane sweeps its four
// nodes as two pairs (nodes 2l, 2l + 1 of each half segment), which keeps
// few registers live; writes go straight from registers, one contiguous run
// per plane and pair.
#pragma once

#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dilbm {

constexpr int TILE_W = 128;   // nodes per row segment (32 lanes x 4 nodes) and per tile row
constexpr int TILE_H = 8;     // rows per binning tile
constexpr int MAXC = 32;      // candidate particles per tile
constexpr int MAXT = 128;     // tiles one particle's phi tail may reach
constexpr int NREC = 3;       // float4 records per binned particle
constexpr int STAGES = 1;     // row segments staged ahead per warp (shared-memory ring depth)
static_assert(STAGES == 1, "a warp carries one staged segment's periodic-edge values (wrap_load)");
constexpr int SWEEP_WARPS = 8;   // default rows in flight per block (one row segment per warp)
constexpr int GUARD = 256;    // elements kept readable before and after a population buffer
constexpr float PHI_CUT_WIDTHS = 4.0f;   // phi tail kept up to 4 interface widths (phi > 1.1e-7)
constexpr unsigned long long WAIT_LIMIT_NS = 1000000000ull;   // bounded device waits: 1 s

enum : int { SIDE_PERIODIC = 0, SIDE_VELOCITY = 1, SIDE_PRESSURE = 2,
             SIDE_HALO = 3 };   // a strip's cut: the rows beyond it come from halo buffers
enum : int { WEST = 0, EAST = 1, SOUTH = 2, NORTH = 3 };
enum : int { ERR_UNSTABLE = 1, ERR_OVERFLOW = 2, ERR_TIMEOUT = 4, ERR_BADPARTICLE = 8 };

// D2Q9 directions of Eq. 3 and weights of Eq. 4.
__host__ __device__ constexpr int cxof(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int cyof(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr float wof(int i) { return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f); }

// ------------------------------------------------------------ storage types
template <typename T> struct Storage;

template <> struct Storage<float> {
    static __device__ __forceinline__ float load1(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float lds1(const float *p) { return *p; }
    static __device__ __forceinline__ void store1(float *p, float v) { *p = v; }
    static __device__ __forceinline__ float2 lds2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ void store2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
};

template <> struct Storage<__half> {
    static __device__ __forceinline__ float load1(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float lds1(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void store1(__half *p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ float2 lds2(const __half *p) { return __half22float2(*reinterpret_cast<const __half2 *>(p)); }
    static __device__ __forceinline__ void store2(__half *p, float2 v) { *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.x, v.y); }
};

template <> struct Storage<__nv_bfloat16> {
    static __device__ __forceinline__ float load1(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float lds1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void store1(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float2 lds2(const __nv_bfloat16 *p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    static __device__ __forceinline__ void store2(__nv_bfloat16 *p, float2 v) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(v.x, v.y);
    }
};

// Elements in the 16-byte halo on each side of a staged row segment, and the
// staged width.
template <typename T> __host__ __device__ constexpr int halo_of() { return 16 / (int)sizeof(T); }
template <typename T> __host__ __device__ constexpr int segw_of() { return TILE_W + 2 * halo_of<T>(); }

// Elements of one stage: the 9 staged rows.
template <typename T> __host__ __device__ constexpr int stage_elems() { return 9 * segw_of<T>(); }

// Dynamic shared memory of one sweep block of W warps.
template <typename T, int W = SWEEP_WARPS> __host__ __device__ constexpr size_t sweep_smem_bytes() {
    return (size_t)W * STAGES * stage_elems<T>() * sizeof(T)   // staged rows
           + (size_t)W * MAXC * NREC * sizeof(float4)           // candidate records
           + (size_t)W * MAXC * sizeof(int)                     // candidate ids
           + (size_t)W * STAGES * sizeof(uint64_t);             // mbarriers
}

// ------------------------------------------------------------ parameters
struct Particles {      // structure of arrays, device memory
    double *x[2], *y[2];        // centre, by step parity
    float *xf[2], *yf[2];       // FP32 copy of the centre, for cheap proximity tests
    double *r, *ux, *uy, *omega, *theta, *rho_s;
    int *fixed;
};

struct Lattice {
    int nx, ny, pitch;          // nodes; row pitch in elements (multiple of 32)
    long long plane;            // elements per population plane (ny * pitch)
    int ntx, nty;               // tiles along x and y
    int per_x, per_y;           // periodic axes
    int wrap_x, wrap_y;         // periodic and short enough that a tile's nodes
                                // need their own minimum image
    int side_kind[4];
    float side_ux[4], side_uy[4], side_drho[4];   // drho = rho_b - 1
    // 16-bit storage holds s_i = (d_i - e_i) / q: d_i = f_i - w_i the FP32
    // deviation, e_i the deviation of the lattice's initial equilibrium
    // f^eq(rho_init, u0) and q a power of two that keeps small s_i out of
    // the FP16 subnormals.  FP32 storage holds d_i itself.
    float ref_e[9];             // e_i
    float ref_q, ref_iq;        // q, 1 / q
    // The moments of the reference e_i (it is the equilibrium deviation of
    // Eq. 2 at rho_init, u0): m0 = rho_init - 1, B = rho_init u0,
    // M = rho_init u0 u0^T (xx, yy, xy), in the moment form below.  The
    // 16-bit sweep takes moments of the stored s_i and adds these, so no
    // per-direction offset enters its inner loop.
    float ref_m[6];
    // A strip of a larger lattice (one rank's rows): the post-collision rows
    // just south (halo[0]) and north (halo[1]) of it, 9 plane rows of `pitch`
    // elements each, with GUARD readable elements before and after; NULL
    // where the side is a physical side of the lattice.
    const void *halo[2];
};

// Is row y of the lattice a south / north edge row (a physical side, not a
// periodic axis and not a strip's cut)?
__host__ __device__ inline bool south_edge_row(const Lattice &L, int y) {
    return !L.per_y && y == 0 && L.side_kind[SOUTH] != SIDE_HALO;
}
__host__ __device__ inline bool north_edge_row(const Lattice &L, int y) {
    return !L.per_y && y == L.ny - 1 && L.side_kind[NORTH] != SIDE_HALO;
}

// Stored value <-> FP32 deviation d_i for direction i (exact scalings by a
// power of two, one rounding in the offset).
template <typename T> __device__ __forceinline__ float from_store(const Lattice &L, int i, float v) {
    if constexpr (std::is_same<T, float>::value) return v;
    else return fmaf(v, L.ref_q, L.ref_e[i]);
}
template <typename T> __device__ __forceinline__ float to_store(const Lattice &L, int i, float d) {
    if constexpr (std::is_same<T, float>::value) return d;
    else return (d - L.ref_e[i]) * L.ref_iq;       // (one rounding: the scaling is exact)
}
struct Physics {
    float omega;                // 1 / tau
    float kf;                   // 1 - 1/(2 tau): prefactor of F_i (Eq. 15)
    float kforce;               // kf (Eq. 18 as printed) or 1 (momentum exchange)
    float phi_k2;               // -4 / (epsilon ln 2): phi = 1 / (1 + 2^(phi_k2 l)) = 1 / (1 + exp(-4 l / eps))
    float cut;                  // phi tail kept while l >= -cut
    int ck;                     // PS: half-width K of each particle's covered-area table (0: none)
    double cut_d;
};

struct Bins {                   // one set per step parity
    int *count;                 // per tile: particles binned (may exceed MAXC)
    int *ids;                   // per tile: MAXC particle ids
    float4 *rec;                // per tile and slot, 3 records: (cx_hi, cx_lo, cy_hi, cy_lo),
                                // (r, ux_hi, uy_hi, omega_hi), (ux_lo, uy_lo, omega_lo, packed
                                // floor(cx), floor(cy): 16 bits each)
    int *pslot;                 // per particle: MAXT entries tile * MAXC + slot (-1: overflowed)
    int *npslot;                // per particle: tiles reached
    float *cover;               // PS: per particle, the covered areas of the (2K+1)^2 cells about
                                // (floor X, floor Y), row-major; shared by both parities
};

// ------------------------------------------------------------ small helpers
__device__ __forceinline__ int wrap_or_clamp(int v, int n, int periodic) {
    if (periodic) return v < 0 ? v + n : (v >= n ? v - n : v);
    return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

// Row sy (in [-1, ny]) of plane i of the post-collision populations `src`:
// wrapped on a periodic axis, from a halo buffer across a strip's cut, else
// clamped (an edge row, whose pulled values the edge scheme replaces).
template <typename T>
__device__ __forceinline__ const T *plane_row(const T *src, const Lattice &L, int i, int sy) {
    if (sy < 0 && L.halo[0]) return static_cast<const T *>(L.halo[0]) + (long long)i * L.pitch;
    if (sy >= L.ny && L.halo[1]) return static_cast<const T *>(L.halo[1]) + (long long)i * L.pitch;
    return src + i * L.plane + (long long)wrap_or_clamp(sy, L.ny, L.per_y) * L.pitch;
}

// Populations of the form X_i = w_i [S + 3 c_i.B + 4.5 c_i^T M c_i] (the
// equilibrium of Eq. 2 has this form with B = rho u, M = rho u u^T; so has the
// collision's relaxation target plus force term of Eqs. 13 and 15), for a
// given zeroth moment m0 = sum_i X_i, so S = m0 - 1.5 tr M.
//
// The constants are chosen so that the moments come out exact for the FP32
// constants themselves: 4.5 w_1 = 1/2 and 4.5 w_5 = 1/8 are exact, the
// first-moment weights a1 ~ 1/3 and a5 = (1 - 2 a1) / 4 satisfy
// 2 a1 + 4 a5 = 1 exactly, and X_0 takes the remainder of m0.  Rounded
// weights would otherwise bias the momentum by ~1e-8 every step.
constexpr float W1F = 1.0f / 9.0f, W5F = 1.0f / 36.0f;
constexpr float A1F = 1.0f / 3.0f;
constexpr float A5F = (float)((1.0 - 2.0 * (double)A1F) / 4.0);

__device__ __forceinline__ void moment_form(float m0, float Bx, float By, float Mxx, float Myy, float Mxy, float X[9]) {
    const float S = fmaf(-1.5f, Mxx + Myy, m0);
    const float ax = fmaf(W1F, S, 0.5f * Mxx), ay = fmaf(W1F, S, 0.5f * Myy);
    const float tr = Mxx + Myy;
    const float ap = fmaf(W5F, S, 0.125f * fmaf(2.0f, Mxy, tr));
    const float am = fmaf(W5F, S, 0.125f * fmaf(-2.0f, Mxy, tr));
    const float bx = A1F * Bx, by = A1F * By, bp = A5F * (Bx + By), bm = A5F * (By - Bx);
    X[0] = fmaf(-2.0f, (ax + ay) + (ap + am), m0);
    X[1] = ax + bx; X[3] = ax - bx;
    X[2] = ay + by; X[4] = ay - by;
    X[5] = ap + bp; X[7] = ap - bp;
    X[6] = am + bm; X[8] = am - bm;
}

// Equilibrium deviation f^eq_i(rho, u) - w_i (Eq. 2), rho = 1 + drho.
__device__ __forceinline__ void eq_dev9(float drho, float rho, float ux, float uy, float X[9]) {
    const float rux = rho * ux, ruy = rho * uy;
    moment_form(drho, rux, ruy, rux * ux, ruy * uy, rux * uy, X);
}

// Collision of Eq. 13 with f^eq of Eq. 2 (corrected velocity, Eq. 17) and the
// force term of Eq. 15, in deviation form:
//   d'_i = d_i + (X_i - omega d_i),  X_i = omega d^eq_i + phi F_i,
// and X has the form w_i [S + 3 c_i.B + 4.5 c_i^T M c_i] with
//   B = omega rho u + k (u_s - u*),  M = omega rho u u^T + k (u_s u_s^T - u* u*^T),
//   sum_i X_i = omega (rho - 1),     k = (1 - 1/2tau) rho phi,
// which is Eqs. 2 and 15 summed and regrouped by powers of c_i.  Because
// rho u = j + phi rho (u_s - u*) / 2 (Eq. 17) and omega/2 + (1 - 1/2tau) = 1,
// B = omega j + phi rho (u_s - u*): the momentum handed to the fluid is formed
// without dividing by rho, so no rounding of j / rho biases it.  The force
// part of M is formed from (u_s - u*) and (u_s + u*) rather than as a
// difference of squares.  Nodes go in pairs on the paired FP32 instructions
// of sm_100+ (each component rounds exactly as the scalar op).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ void moment_form2(float2 m0, float2 Bx, float2 By, float2 Mxx, float2 Myy, float2 Mxy,
                                             float2 X[9]) {
    const float2 tr = add2(Mxx, Myy);
    const float2 S = fma2(f2(-1.5f), tr, m0);
    const float2 ax = fma2(f2(W1F), S, mul2(f2(0.5f), Mxx)), ay = fma2(f2(W1F), S, mul2(f2(0.5f), Myy));
    const float2 ap = fma2(f2(W5F), S, mul2(f2(0.125f), fma2(f2(2.0f), Mxy, tr)));
    const float2 am = fma2(f2(W5F), S, mul2(f2(0.125f), fma2(f2(-2.0f), Mxy, tr)));
    const float2 bx = mul2(f2(A1F), Bx), by = mul2(f2(A1F), By);
    const float2 bp = mul2(f2(A5F), add2(Bx, By)), bm = mul2(f2(A5F), sub2(By, Bx));
    X[0] = fma2(f2(-2.0f), add2(add2(ax, ay), add2(ap, am)), m0);
    X[1] = add2(ax, bx); X[3] = sub2(ax, bx);
    X[2] = add2(ay, by); X[4] = sub2(ay, by);
    X[5] = add2(ap, bp); X[7] = sub2(ap, bp);
    X[6] = add2(am, bm); X[8] = sub2(am, bm);
}

// d + (X - omega d): the small change is rounded on its own before it is
// added (a single fma((1 - omega), d, X) measured ~15% larger errors against
// the FP64 oracle on wall-driven flow).
__device__ __forceinline__ void relax2(float2 d[9], float omega, const float2 X[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = add2(d[i], fma2(f2(-omega), d[i], X[i]));
}

// The collision acts on the stored values.  FP32 stores d_i itself.  16-bit
// storage holds s_i = (d_i - e_i) / q, and since e_i has the moment form
// with the reference moments (m0e, Be, Me) and q is a power of two,
//   s'_i = s_i + (Y_i - omega s_i),  Y = (X - omega e) / q,
// where Y is the moment form of (omega sum s, (B - omega Be) / q,
// (M - omega Me) / q): the zeroth input is omega times the stored values'
// own sum, the first moment's part omega j becomes omega times the stored
// first moment, and only M, a product of the physical moments, needs the
// reference subtracted.  (ms, jxs, jys are the moments of the stored values.)
template <typename T>
__device__ __forceinline__ void relax_to2(float2 d[9], const Lattice &L, float omega, float2 ms, float2 Bxs,
                                          float2 Bys, float2 Mxx, float2 Myy, float2 Mxy) {
    const float2 om = f2(omega);
    if constexpr (!std::is_same<T, float>::value) {
        const float2 iq = f2(L.ref_iq);
        Mxx = mul2(sub2(Mxx, f2(omega * L.ref_m[3])), iq);
        Myy = mul2(sub2(Myy, f2(omega * L.ref_m[4])), iq);
        Mxy = mul2(sub2(Mxy, f2(omega * L.ref_m[5])), iq);
    }
    float2 X[9];
    moment_form2(mul2(om, ms), Bxs, Bys, Mxx, Myy, Mxy, X);
    relax2(d, omega, X);
}

// phi = 0 (plain BGK of Eq. 1): B = omega j and, as rho u = j,
// M = omega rho u u^T = B u^T.
template <typename T>
__device__ __forceinline__ void collide_plain2(float2 d[9], const Lattice &L, float omega, float2 ms, float2 jxs,
                                               float2 jys, float2 jx, float2 jy, float2 ux, float2 uy) {
    const float2 om = f2(omega);
    const float2 Bx = mul2(om, jx), By = mul2(om, jy);
    if constexpr (std::is_same<T, float>::value)
        relax_to2<T>(d, L, omega, ms, Bx, By, mul2(Bx, ux), mul2(By, uy), mul2(Bx, uy));
    else
        relax_to2<T>(d, L, omega, ms, mul2(om, jxs), mul2(om, jys), mul2(Bx, ux), mul2(By, uy), mul2(Bx, uy));
}

template <typename T>
__device__ __forceinline__ void collide2(float2 d[9], const Lattice &L, float omega, float2 ms, float2 jxs,
                                         float2 jys, float2 rho, float2 ux, float2 uy, float2 kphi, float2 prho,
                                         float2 dux, float2 duy, float2 usx, float2 usy, float2 uax, float2 uay) {
    const float2 om = f2(omega);
    const float2 orho = mul2(om, rho);
    float2 px = mul2(prho, dux), py = mul2(prho, duy);
    if constexpr (!std::is_same<T, float>::value) {
        px = mul2(px, f2(L.ref_iq));
        py = mul2(py, f2(L.ref_iq));
    }
    const float2 Bxs = fma2(om, jxs, px), Bys = fma2(om, jys, py);
    const float2 rux = mul2(orho, ux);
    const float2 Mxx = fma2(rux, ux, mul2(kphi, mul2(dux, add2(usx, uax))));
    const float2 Myy = fma2(mul2(orho, uy), uy, mul2(kphi, mul2(duy, add2(usy, uay))));
    const float2 Mxy = fma2(rux, uy, mul2(kphi, fma2(dux, usy, mul2(uax, duy))));
    relax_to2<T>(d, L, omega, ms, Bxs, Bys, Mxx, Myy, Mxy);
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

// ------------------------------------------------------------ async copies
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for a phase of an mbarrier, giving up after WAIT_LIMIT_NS.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
}

// Order this thread's earlier shared-memory reads before later writes of the
// async proxy (the bulk copies) to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Stage the nine source rows of row segment (row y, segment tx):
// plane i comes from row y - c_iy, columns [tx*128 - halo, tx*128 + 128 + halo).
// Lane 0 arms the barrier with the byte count, lanes 0..8 issue one copy each.
// The population buffers carry GUARD readable elements before and after, so
// the copies of edge segments stay inside the allocation.
template <typename T>
__device__ __forceinline__ void issue_segment(const T *__restrict__ src, const Lattice &L, int y, int tx, T *stage,
                                              uint64_t *bar, int lane) {
    constexpr int H = halo_of<T>(), SW = segw_of<T>();
    if (lane == 0) mbar_expect_tx(bar, 9u * SW * sizeof(T));
    __syncwarp();
    if (lane < 9) {
        const T *g = plane_row<T>(src, L, lane, y - cyof(lane)) + (tx * TILE_W - H);
        bulk_copy_g2s(stage + lane * SW, g, SW * sizeof(T), bar);
    }
}

// Periodic x: the staged halo of a row's first segment does not hold column
// nx - 1 (what node 0 streams from in the three directions with c_ix = +1),
// nor does the stage of its last segment hold column 0 after column nx - 1
// (what node nx - 1 streams from with c_ix = -1).  When a warp issues such a
// segment's copy, lanes 0..2 also load the first value (planes 1, 5, 8) and
// lanes 3..5 the second (planes 3, 6, 7), raw; once the copy has landed,
// wrap_patch writes them where the pulls look.  wrap_lane_plane gives the
// plane of the lane's value and whether the segment needs it.
__device__ __forceinline__ int wrap_lane_plane(const Lattice &L, int tx, int lane) {
    if (!L.per_x || lane >= 6) return -1;
    const bool first = tx == 0, last = tx * TILE_W + TILE_W >= L.nx;
    if (lane < 3) return first ? (lane == 0 ? 1 : (lane == 1 ? 5 : 8)) : -1;
    return last ? (lane == 3 ? 3 : (lane == 4 ? 6 : 7)) : -1;
}

template <typename T>
__device__ __forceinline__ T wrap_load(const T *__restrict__ src, const Lattice &L, int y, int tx, int lane) {
    const int i = wrap_lane_plane(L, tx, lane);
    if (i < 0) return T();
    const T *row = plane_row<T>(src, L, i, y - cyof(i));
    return row[lane < 3 ? L.nx - 1 : 0];
}

template <typename T>
__device__ __forceinline__ void wrap_patch(T *stage, const Lattice &L, int tx, int lane, T v) {
    constexpr int H = halo_of<T>(), SW = segw_of<T>();
    const int i = wrap_lane_plane(L, tx, lane);
    if (i >= 0) stage[i * SW + (lane < 3 ? H - 1 : H + (L.nx - tx * TILE_W))] = v;
}

template <typename T>
__device__ __forceinline__ void pull_node_scalar(const T *__restrict__ src, const Lattice &L, int x, int y, float d[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sx = wrap_or_clamp(x - cxof(i), L.nx, L.per_x);
        d[i] = from_store<T>(L, i, Storage<T>::load1(plane_row<T>(src, L, i, y - cyof(i)) + sx));
    }
}

// Non-equilibrium extrapolation at an edge node (x, y) (Guo et al. 2002, as
// the paper's Sec. 3 uses): d_b = deq(rho_b, u_b) + d_n - deq(rho_n, u_n),
// with n the inner neighbour (diagonal at corners; corners take the
// south/north condition).  Kept out of line: few nodes take it, and inlined
// it would crowd the sweep's instruction cache.
struct Pop9 {
    float v[9];
};

// d_b from the inner neighbour's streamed values dn and the side's condition.
__device__ __forceinline__ void extrapolate(const Lattice &L, int side, const float dn[9], float out[9]) {
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
    // f^eq(rho_b, u_b) - f^eq(rho_n, u_n) is linear in the moments, so it is
    // the moment form of the moment differences, formed without cancellation:
    // with d = rho_b - rho_n and v = u_b - u_n,
    //   rho_b u_b - rho_n u_n = d u_b + rho_n v,
    //   rho_b u_b u_b - rho_n u_n u_n = d u_b u_b + rho_n (v (u_b + u_n))   (xx, yy),
    //   rho_b ubx uby - rho_n unx uny = d ubx uby + rho_n (vx uby + unx vy).
    const float d = drb - drn, vx = ubx - unx, vy = uby - uny;
    const float Bx = fmaf(d, ubx, rhon * vx), By = fmaf(d, uby, rhon * vy);
    const float Mxx = fmaf(d * ubx, ubx, rhon * (vx * (ubx + unx)));
    const float Myy = fmaf(d * uby, uby, rhon * (vy * (uby + uny)));
    const float Mxy = fmaf(d * ubx, uby, rhon * fmaf(vx, uby, unx * vy));
    float X[9];
    moment_form(d, Bx, By, Mxx, Myy, Mxy, X);
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i] = dn[i] + X[i];
}

// An edge node whose inner neighbour lies on another row (south / north
// edges and corners): the neighbour's streamed values come from global memory.
template <typename T>
__device__ __noinline__ Pop9 edge_values(const T *__restrict__ src, const Lattice &L, int x, int y) {
    const int onx = !L.per_x && (x == 0 || x == L.nx - 1);
    const int ony = south_edge_row(L, y) || north_edge_row(L, y);
    const int side = ony ? (y == 0 ? SOUTH : NORTH) : (x == 0 ? WEST : EAST);
    const int xn = onx ? (x == 0 ? 1 : L.nx - 2) : x;
    const int yn = ony ? (y == 0 ? 1 : L.ny - 2) : y;
    float dn[9];
    pull_node_scalar<T>(src, L, xn, yn, dn);
    Pop9 out;
    extrapolate(L, side, dn, out.v);
    return out;
}

// ------------------------------------------------------------ PS-LBM solid fraction
// The paper's comparison method (PS-LBM, Sec. 2.2) weights its collision by
// B = eps_s (Eq. 8), the area of the node's unit cell covered by the solid.
// cell_cover returns the area of [dx - 1/2, dx + 1/2] x [dy - 1/2, dy + 1/2]
// inside the disc of radius r >= 1 centred at the origin: the shoelace area
// of the polygon formed, counter-clockwise, by the corners inside the disc
// and the points where the circle crosses the cell edges, plus the circular
// segment between each chord that polygon draws across the circle and its
// arc.  The polygon is summed in the cell's own frame (coordinates of size
// 1/2, so FP32 keeps ~1e-6).  Each corner is classified once (inside:
// distance < r) and every edge takes its crossings from the classes of its
// two ends (one crossing where they differ; none or two where both are
// outside), so a corner on the circle, seen by two edges, cannot be counted
// twice or lost.  For r >= 1 every arc inside a unit cell is a minor arc.
// Both routines stay out of line: inlined into the sweep's four node slots
// they evict the sweep's own code from the instruction cache.
static __device__ __noinline__ float segment_area(float ex, float ey, float ix, float iy, float r, float rinv) {
    // area between the chord E-I and the minor arc: r^2 (asin s - s sqrt(1 - s^2)), s = |EI| / 2r
    const float s = 0.5f * sqrtf((ix - ex) * (ix - ex) + (iy - ey) * (iy - ey)) * rinv;
    float g;
    if (s < 0.3f) {     // Taylor series: 2/3 s^3 + 1/5 s^5 + 3/28 s^7 + 5/72 s^9 + 35/704 s^11
        const float s2 = s * s;
        g = s * s2 * (2.0f / 3.0f + s2 * (0.2f + s2 * (3.0f / 28.0f + s2 * (5.0f / 72.0f + s2 * (35.0f / 704.0f)))));
    } else {
        g = asinf(s) - s * sqrtf((1.0f - s) * (1.0f + s));
    }
    return r * r * g;
}

// The polygon and segment sums of cell_cover, fed one boundary point at a
// time in counter-clockwise order.
struct CoverWalk {
    float r, rinv;
    float area2 = 0.f, seg = 0.f;
    float fx = 0.f, fy = 0.f, lx = 0.f, ly = 0.f;   // first and last polygon vertex
    float ex = 0.f, ey = 0.f, ix0 = 0.f, iy0 = 0.f; // pending exit; first entry seen before any exit
    bool any = false, pending = false, first_entry = false;

    __device__ __forceinline__ void vertex(float vx, float vy) {
        if (any) area2 += lx * vy - vx * ly;
        else { fx = vx; fy = vy; any = true; }
        lx = vx; ly = vy;
    }
    __device__ __forceinline__ void entry(float vx, float vy) {
        if (pending) { seg += segment_area(ex, ey, vx, vy, r, rinv); pending = false; }
        else if (!first_entry) { first_entry = true; ix0 = vx; iy0 = vy; }
        vertex(vx, vy);
    }
    __device__ __forceinline__ void exit(float vx, float vy) {
        vertex(vx, vy);
        ex = vx; ey = vy; pending = true;
    }
};

// Half the chord the circle cuts on a line at distance |p| from the centre.
__device__ __forceinline__ float half_chord(float p, float r) {
    const float a = fabsf(p);
    return sqrtf(fmaxf((r - a) * (r + a), 0.f));
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

static __device__ __noinline__ float cell_cover(float dx, float dy, float r) {
    // the cell's extent about the disc centre; corners 0..3 counter-clockwise
    // from (x0, y0), edge k from corner k to corner k + 1
    const float x0 = dx - 0.5f, x1 = dx + 0.5f, y0 = dy - 0.5f, y1 = dy + 0.5f;
    const float r2 = r * r;
    const float xx0 = x0 * x0, xx1 = x1 * x1, yy0 = y0 * y0, yy1 = y1 * y1;
    const bool in0 = xx0 + yy0 < r2, in1 = xx1 + yy0 < r2, in2 = xx1 + yy1 < r2, in3 = xx0 + yy1 < r2;
    // both ends outside: the circle crosses twice iff the foot of the
    // perpendicular from the centre lies inside the edge and |p| < r
    const bool mx = x0 < 0.f && 0.f < x1, my = y0 < 0.f && 0.f < y1;
    CoverWalk w;
    w.r = r;
    w.rinv = __frcp_rn(r);

    // edge 0: y = y0, x rising; enters at x = -h, leaves at x = +h
    if (in0) w.vertex(-0.5f, -0.5f);
    {
        const bool two = !in0 && !in1 && mx && fabsf(y0) < r;
        const bool en = !in0 && (in1 || two), ex = !in1 && (in0 || two);
        if (en || ex) {
            const float h = half_chord(y0, r);
            if (en) w.entry(clampf(-h, x0, x1) - dx, -0.5f);
            if (ex) w.exit(clampf(h, x0, x1) - dx, -0.5f);
        }
    }
    // edge 1: x = x1, y rising; enters at y = -h, leaves at y = +h
    if (in1) w.vertex(0.5f, -0.5f);
    {
        const bool two = !in1 && !in2 && my && fabsf(x1) < r;
        const bool en = !in1 && (in2 || two), ex = !in2 && (in1 || two);
        if (en || ex) {
            const float h = half_chord(x1, r);
            if (en) w.entry(0.5f, clampf(-h, y0, y1) - dy);
            if (ex) w.exit(0.5f, clampf(h, y0, y1) - dy);
        }
    }
    // edge 2: y = y1, x falling; enters at x = +h, leaves at x = -h
    if (in2) w.vertex(0.5f, 0.5f);
    {
        const bool two = !in2 && !in3 && mx && fabsf(y1) < r;
        const bool en = !in2 && (in3 || two), ex = !in3 && (in2 || two);
        if (en || ex) {
            const float h = half_chord(y1, r);
            if (en) w.entry(clampf(h, x0, x1) - dx, 0.5f);
            if (ex) w.exit(clampf(-h, x0, x1) - dx, 0.5f);
        }
    }
    // edge 3: x = x0, y falling; enters at y = +h, leaves at y = -h
    if (in3) w.vertex(-0.5f, 0.5f);
    {
        const bool two = !in3 && !in0 && my && fabsf(x0) < r;
        const bool en = !in3 && (in0 || two), ex = !in0 && (in3 || two);
        if (en || ex) {
            const float h = half_chord(x0, r);
            if (en) w.entry(-0.5f, clampf(h, y0, y1) - dy);
            if (ex) w.exit(-0.5f, clampf(-h, y0, y1) - dy);
        }
    }
    if (!w.any) return 0.f;
    w.area2 += w.lx * w.fy - w.fx * w.ly;
    if (w.pending && w.first_entry) w.seg += segment_area(w.ex, w.ey, w.ix0, w.iy0, r, w.rinv);
    return 0.5f * w.area2 + w.seg;
}

// ------------------------------------------------------------ the sweep
// Mode: STEP writes the collided populations and the force partials; FIELDS
// writes rho, the corrected velocity and phi of the streamed state instead.
enum : int { MODE_STEP = 0, MODE_FIELDS = 1 };

struct FieldsOut {
    float *rho, *ux, *uy, *phi;   // dense [ny][nx]
};

// Everything one lattice's sweep needs.
template <typename T>
struct SweepArgs {
    const T *src;               // post-collision populations (GUARD elements in)
    T *dst;                     // next populations
    Lattice L;
    Physics ph;
    Bins B;                     // this step's bins (counts, ids, records)
    float4 *partial;            // force / torque partials
    int *clear;                 // next step's bin counts to zero, or NULL
    int *err;                   // the lattice's error word
    FieldsOut fo;               // MODE_FIELDS outputs
};

// A batched sweep walks one work list over many lattices, their descriptors
// held in the kernel's parameter space (uniform constant-cache reads, no
// aliasing with the stores): lattice k owns row segments
// [item_start[k], item_start[k+1]) and tiles [tile_start[k], tile_start[k+1]).
constexpr int BATCH_LAUNCH_MAX = 84;     // lattices per batched launch

template <typename T>
struct BatchArgs {
    SweepArgs<T> a[BATCH_LAUNCH_MAX];
    int item_start[BATCH_LAUNCH_MAX + 1];
    int tile_start[BATCH_LAUNCH_MAX + 1];
    int n;
};
static_assert(sizeof(BatchArgs<float>) <= 32000, "batched sweep parameters exceed the parameter space");

// Particle batches keep their descriptors in device memory: lattice k owns
// particles [item_start[k], item_start[k+1]).
struct BatchIndex {
    const int *item_start;
    const int *tile_start;
    int n;
};

// Largest k with start[k] <= v (start[0] = 0, start ascending, n entries + 1).
template <typename P>
__device__ __forceinline__ int batch_find(const P &start, int n, int v) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Per-warp state of the staging ring.
struct Ring {
    uint64_t *bars;
    uint32_t parity;            // bit s: phase parity the next wait on stage s expects
    uint32_t pending;           // bit s: stage s has copies in flight
};

// The streamed value f_i(x) = f'_i(x - c_i) of plane i at node e of the
// staged segment (e in [-1, TILE_W]: the 16-byte halos hold the neighbours).
template <typename T, int I>
__device__ __forceinline__ float staged_pull(const Lattice &L, const T *stage, int e) {
    constexpr int H = halo_of<T>(), SW = segw_of<T>();
    return from_store<T>(L, I, Storage<T>::lds1(stage + I * SW + H + e - cxof(I)));
}

template <typename T, int I = 0>
__device__ __forceinline__ void staged_pull9(const Lattice &L, const T *stage, int e, float out[9]) {
    out[I] = staged_pull<T, I>(L, stage, e);
    if constexpr (I < 8) staged_pull9<T, I + 1>(L, stage, e, out);
}

// The hardware's base-2 exponential and reciprocal (PTX ex2.approx, rcp.approx;
// subnormal results flush to zero, so 2^x for very negative x is 0).
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Slot m (0 or 1) of a node pair.
__device__ __forceinline__ float &slot(float2 &v, int m) { return m ? v.y : v.x; }

// One row segment (row y, segment tx) of lattice A: wait for its staged rows
// (and write in the periodic-edge values wv, see wrap_load), then sweep its
// 128 nodes in two passes of 64 (lane l takes nodes 2l and 2l + 1 of each
// half, so every store of a pass is one contiguous run per plane), hand the
// stage to the segment `nxt` (row ny2, segment nx2 of lattice An; its edge
// values go to wv) once the second pass has read it, and sum the segment's
// force / torque per candidate particle.  Returns false if the bounded wait
// gave up.
template <typename T, int MODE, bool EDGES, bool PS = false>
__device__ __forceinline__ bool sweep_segment(const SweepArgs<T> &A, int y, int tx, T *stage, Ring &ring, int s,
                                              bool has_next, const SweepArgs<T> &An, int ny2, int nx2,
                                              float4 *crec, int *cid, T &wv, int lane) {
    constexpr int H = halo_of<T>(), SW = segw_of<T>();
    const Lattice &L = A.L;
    const Physics &ph = A.ph;
    const int ty = y / TILE_H, tile = ty * L.ntx + tx;
    const int tx0 = tx * TILE_W, ty0 = ty * TILE_H;

    // ---- the tile's candidate particles (records written by the binning),
    // loaded before the wait so that their latency overlaps it
    __syncwarp();
    int ncand = 0;
    if (A.B.count) {
        ncand = A.B.count[tile];
        ncand = ncand > MAXC ? MAXC : ncand;
        if (lane < ncand) {
            const long long r = (long long)tile * MAXC + lane;
#pragma unroll
            for (int q = 0; q < NREC; ++q) crec[q * MAXC + lane] = A.B.rec[NREC * r + q];
            cid[lane] = A.B.ids[r];
        }
    }

    // ---- wait for the staged rows
    // a warp-uniform decision: every lane leaves together if any gave up
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&ring.bars[s], (ring.parity >> s) & 1u))) return false;
    ring.parity ^= 1u << s;
    ring.pending &= ~(1u << s);

    const bool row_edge = EDGES && (south_edge_row(L, y) || north_edge_row(L, y));
    const bool col_edge = EDGES && !L.per_x && (tx == 0 || tx0 + TILE_W >= L.nx);
    if (L.per_x && (tx == 0 || tx0 + TILE_W >= L.nx)) wrap_patch<T>(stage, L, tx, lane, wv);
    // west / east edge nodes of a row that is not itself an edge row: the
    // non-equilibrium extrapolation from the inner neighbour's streamed values
    // (same row, staged).  Pull streaming reads each staged value at exactly
    // one node, so in FP32 storage lane 0 (west) and lane 1 (east) write the
    // edge node's extrapolated populations into the cells that node's pulls
    // read, and the pulls below pick them up.  (For nx >= 3 the cells one
    // edge writes and those the other reads are distinct.)  16-bit storage
    // would round them on the way; there the passes replace the pulled values.
    constexpr bool EDGE_IN_STAGE = std::is_same<T, float>::value;
    if (EDGE_IN_STAGE && col_edge && !row_edge && lane < 2) {
        const int xm = lane == 0 ? 0 : L.nx - 1;
        const int e = xm - tx0;
        if (e >= 0 && e < TILE_W) {
            float dn[9], ev[9];
            staged_pull9<T>(L, stage, e + (lane == 0 ? 1 : -1), dn);
            extrapolate(L, lane == 0 ? WEST : EAST, dn, ev);
#pragma unroll
            for (int i = 0; i < 9; ++i) Storage<T>::store1(stage + i * SW + H + e - cxof(i), to_store<T>(L, i, ev[i]));
        }
    }
    __syncwarp();   // candidate records and edge values visible to the whole warp

    // lane c < ncand: the segment's force / torque on candidate c so far
    // (first pass, then second pass added)
    float sgx = 0.f, sgy = 0.f, sgt = 0.f;
    unsigned badmax = 0u;

    // a row's last segment may end within its first half: its second pass
    // would hold no node (no store, no force share), so it is not run
    const int npass = tx0 + TILE_W / 2 < L.nx ? 2 : 1;
#pragma unroll 1
    for (int pass = 0; pass < npass; ++pass) {
        const int e = pass * (TILE_W / 2) + 2 * lane;    // the pair's first node within the segment
        const int x = tx0 + e;

        // ---- pull-stream from the staged rows: f_i(x, t+1) = f'_i(x - c_i, t)
        float2 dk[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const T *row = stage + i * SW + H + e;
            if (cxof(i) == 0) dk[i] = Storage<T>::lds2(row);
            else dk[i] = make_float2(Storage<T>::lds1(row - cxof(i)), Storage<T>::lds1(row + 1 - cxof(i)));
        }
        if constexpr (!EDGE_IN_STAGE) {
            if (col_edge && !row_edge) {
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int xm = x + m;
                    if (xm != 0 && xm != L.nx - 1) continue;
                    float dn[9], ev[9];
                    staged_pull9<T>(L, stage, e + m + (xm == 0 ? 1 : -1), dn);
                    extrapolate(L, xm == 0 ? WEST : EAST, dn, ev);
#pragma unroll
                    for (int i = 0; i < 9; ++i) slot(dk[i], m) = to_store<T>(L, i, ev[i]);
                }
            }
        }
        // the segment's last reads of the stage are done: recycle it for the
        // segment STAGES items ahead
        if (pass == npass - 1) {
            __syncwarp();
            if (has_next) {
                fence_proxy_async_smem();
                issue_segment<T>(An.src, An.L, ny2, nx2, stage, &ring.bars[s], lane);
                wv = wrap_load<T>(An.src, An.L, ny2, nx2, lane);
                ring.pending |= 1u << s;
            }
        }
        if (EDGES && row_edge) {
            // south / north edge rows (corners included): neighbour on another row
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                if (x + m >= L.nx) continue;
                const Pop9 ev = edge_values<T>(A.src, L, x + m, y);
#pragma unroll
                for (int i = 0; i < 9; ++i) slot(dk[i], m) = to_store<T>(L, i, ev.v[i]);
            }
        }

        // ---- solid fraction (Eq. 14), owner and particle velocity per node:
        // max over the tile's candidates, lowest particle id on ties
        float phi[2] = {0.f, 0.f}, rxn[2] = {0.f, 0.f}, ryn[2] = {0.f, 0.f};
        int best[2] = {-1, -1}, best_id[2] = {0x7fffffff, 0x7fffffff};
        // (ncand is warp-uniform; a segment no particle reaches skips all of it)
        for (int c = 0; c < ncand; ++c) {
            const float4 ra = crec[c], rb = crec[MAXC + c];
            const float R = rb.x + ph.cut;
            float dy = ((float)(y - ty0) - ra.z) - ra.w;
            // short periodic axes: the stored image may lie several periods away
            // (it is the one nearest the tile centre), so reduce by the nearest
            // multiple of the period (exact: an integer multiple of an integer)
            int ky = 0;                                     // PS: periods removed, for the table index
            if (L.wrap_y) {
                const float k = rintf(dy * __frcp_rn((float)L.ny));
                dy = fmaf(-(float)L.ny, k, dy);
                ky = (int)k;
            }
            const float h2 = fmaf(-dy, dy, R * R);
            if (h2 < 0.f) continue;                         // this row misses the disc tail
            const float dx0 = ((float)e - ra.x) - ra.y;
            if (!L.wrap_x) {
                // the pair spans [dx0, dx0 + 1]
                const float lo = dx0 > 0.f ? dx0 : (dx0 + 1.0f < 0.f ? -(dx0 + 1.0f) : 0.f);
                if (lo * lo > h2) continue;
            }
            const int id = cid[c];
            if constexpr (PS) {
                // covered cell fraction (B = eps_s, Eq. 8): 1 once every corner is
                // inside, else the particle's table entry for the cell.  Both
                // nodes' entries are fetched before either is used.  The
                // centre's whole-cell offsets come packed in the record.
                const int fpk = __float_as_int(crec[2 * MAXC + c].w);
                const int K = ph.ck, S = 2 * K + 1;
                const float *tab = A.B.cover + (long long)id * S * S;
                const int iy = (y - ty0) - (int)(short)((unsigned)fpk >> 16) - L.ny * ky + K;
                float pcq[2], dxq[2];
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    float dx = dx0 + (float)m;
                    int kx = 0;
                    if (L.wrap_x) {
                        const float k = rintf(dx * __frcp_rn((float)L.nx));
                        dx = fmaf(-(float)L.nx, k, dx);
                        kx = (int)k;
                    }
                    dxq[m] = dx;
                    const float d2 = fmaf(dx, dx, dy * dy);
                    const float l = rb.x - sqrtf(d2);
                    const int ix = e + m - (int)(short)(fpk & 0xffff) - L.nx * kx + K;
                    const bool inside = d2 <= R * R && l >= -ph.cut;
                    const bool look = inside && l < ph.cut && (unsigned)ix < (unsigned)S && (unsigned)iy < (unsigned)S;
                    pcq[m] = look ? __ldg(tab + iy * S + ix) : (inside && l >= ph.cut ? 1.0f : 0.f);
                }
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const float pc = pcq[m];
                    if (!(pc > 0.f)) continue;
                    if (pc > phi[m] || (pc == phi[m] && id < best_id[m])) {
                        phi[m] = pc; best[m] = c; best_id[m] = id; rxn[m] = dxq[m]; ryn[m] = dy;
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    float dx = dx0 + (float)m;
                    if (L.wrap_x) dx = fmaf(-(float)L.nx, rintf(dx * __frcp_rn((float)L.nx)), dx);
                    const float d2 = fmaf(dx, dx, dy * dy);
                    if (d2 > R * R) continue;
                    const float l = rb.x - sqrtf(d2);
                    if (l < -ph.cut) continue;
                    // (1 + tanh(2l/eps)) / 2 == 1 / (1 + exp(-4l/eps)) == 1 / (1 + 2^(phi_k2 l)),
                    // with the hardware's base-2 exponential and reciprocal: the
                    // rounding of the argument phi_k2 l (|.| <= 23 inside the tail,
                    // a relative error of at most 23 * 2^-24 in the power) bounds
                    // the error either way, and both instructions add about an ulp
                    const float pc = rcp_approx(1.0f + ex2_approx(ph.phi_k2 * l));
                    if (pc > phi[m] || (pc == phi[m] && pc > 0.f && id < best_id[m])) {
                        phi[m] = pc; best[m] = c; best_id[m] = id; rxn[m] = dx; ryn[m] = dy;
                    }
                }
            }
        }

        // warps with no node inside any particle's phi tail collide without the force term
        const bool coupled = ncand > 0 && __any_sync(0xffffffffu, max(best[0], best[1]) >= 0);
        const bool act_a = x < L.nx, act_b = x + 1 < L.nx;

        // ---- moments (Eq. 5, Eq. 16): of the stored values, then physical
        const float2 ms = add2(add2(add2(add2(dk[0], dk[1]), add2(dk[2], dk[3])),
                                    add2(add2(dk[4], dk[5]), add2(dk[6], dk[7]))), dk[8]);
        const float2 jxs = add2(add2(sub2(dk[1], dk[3]), sub2(dk[5], dk[6])), sub2(dk[8], dk[7]));
        const float2 jys = sub2(add2(sub2(dk[2], dk[4]), add2(dk[5], dk[6])), add2(dk[7], dk[8]));
        float2 drho = ms, jx = jxs, jy = jys;
        if constexpr (!std::is_same<T, float>::value) {
            const float2 q = f2(L.ref_q);
            drho = fma2(q, ms, f2(L.ref_m[0]));
            jx = fma2(q, jxs, f2(L.ref_m[1]));
            jy = fma2(q, jys, f2(L.ref_m[2]));
        }
        const float2 rho = add2(f2(1.0f), drho);
        // u* (Eq. 16); CUDA's correctly rounded reciprocal (a biased one would
        // bias u* the same way on every node and step)
        const float2 inv = make_float2(__frcp_rn(rho.x), __frcp_rn(rho.y));
        const float2 ua = mul2(jx, inv), va = mul2(jy, inv);
        if (MODE == MODE_STEP) {
            // unstable: rho <= 0 or not finite (a non-finite population makes
            // rho non-finite); as unsigned, bits(rho) - 1 exceeds the largest
            // finite float's bits - 1 exactly then
            badmax = max(badmax, act_a ? __float_as_uint(rho.x) - 1u : 0u);
            badmax = max(badmax, act_b ? __float_as_uint(rho.y) - 1u : 0u);
        }

        if (!coupled) {
            if (MODE == MODE_FIELDS) {
                const long long o = (long long)y * L.nx + x;
                if (act_a) {
                    if (A.fo.rho) A.fo.rho[o] = rho.x;
                    if (A.fo.ux) A.fo.ux[o] = ua.x;
                    if (A.fo.uy) A.fo.uy[o] = va.x;
                    if (A.fo.phi) A.fo.phi[o] = 0.f;
                }
                if (act_b) {
                    if (A.fo.rho) A.fo.rho[o + 1] = rho.y;
                    if (A.fo.ux) A.fo.ux[o + 1] = ua.y;
                    if (A.fo.uy) A.fo.uy[o + 1] = va.y;
                    if (A.fo.phi) A.fo.phi[o + 1] = 0.f;
                }
                continue;
            }
            collide_plain2<T>(dk, L, ph.omega, ms, jxs, jys, jx, jy, ua, va);
        } else {
            // u_s - u* from the particle velocity carried as FP32 hi + lo:
            // u_s = U + omega x r with r the node's offset from the centre
            float du[2] = {0.f, 0.f}, dv[2] = {0.f, 0.f};
            const float uas[2] = {ua.x, ua.y}, vas[2] = {va.x, va.y};
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int b = best[m];
                if (b >= 0) {
                    const float4 rb = crec[MAXC + b], rl = crec[2 * MAXC + b];
                    du[m] = fmaf(-rb.w, ryn[m], rb.y - uas[m]) + fmaf(-rl.z, ryn[m], rl.x);
                    dv[m] = fmaf(rb.w, rxn[m], rb.z - vas[m]) + fmaf(rl.z, rxn[m], rl.y);
                }
            }
            const float2 dux = make_float2(du[0], du[1]), duy = make_float2(dv[0], dv[1]);
            const float2 usx = add2(ua, dux), usy = add2(va, duy);
            const float2 phq = make_float2(phi[0], phi[1]);
            // ---- corrected velocity (Eq. 17)
            // (PS-LBM: f^eq takes the fluid velocity u*, there is no correction)
            const float2 hph = mul2(f2(PS ? 0.0f : 0.5f), phq);
            const float2 ux = fma2(hph, dux, ua), uy = fma2(hph, duy, va);

            if (MODE == MODE_FIELDS) {
                const long long o = (long long)y * L.nx + x;
                if (act_a) {
                    if (A.fo.rho) A.fo.rho[o] = rho.x;
                    if (A.fo.ux) A.fo.ux[o] = ux.x;
                    if (A.fo.uy) A.fo.uy[o] = uy.x;
                    if (A.fo.phi) A.fo.phi[o] = phq.x;
                }
                if (act_b) {
                    if (A.fo.rho) A.fo.rho[o + 1] = rho.y;
                    if (A.fo.ux) A.fo.ux[o + 1] = ux.y;
                    if (A.fo.uy) A.fo.uy[o + 1] = uy.y;
                    if (A.fo.phi) A.fo.phi[o + 1] = phq.y;
                }
                continue;
            }
            const float2 prho = mul2(rho, phq);
            collide2<T>(dk, L, ph.omega, ms, jxs, jys, rho, ux, uy, mul2(f2(ph.kf), prho), prho, dux, duy, usx, usy,
                        ua, va);

            // ---- Eqs. 18-19 per node, by the closed form sum_i F_i c_i = kf rho (u_s - u*),
            // summed per candidate over the pass (the lane's two nodes, then a
            // fixed shuffle tree) and added to that candidate's lane
            const int own_a = act_a ? best[0] : -1, own_b = act_b ? best[1] : -1;
            const float sa = -prho.x * ph.kforce, sb = -prho.y * ph.kforce;
            const float gax = sa * du[0], gay = sa * dv[0], gbx = sb * du[1], gby = sb * dv[1];
            const float ta = fmaf(rxn[0], gay, -(ryn[0] * gax)), tb = fmaf(rxn[1], gby, -(ryn[1] * gbx));
            for (int c = 0; c < ncand; ++c) {
                float v0 = 0.f, v1 = 0.f, v2 = 0.f;
                if (own_a == c) { v0 = gax; v1 = gay; v2 = ta; }
                if (own_b == c) { v0 += gbx; v1 += gby; v2 += tb; }
                if (!__any_sync(0xffffffffu, own_a == c || own_b == c)) continue;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                    v2 += __shfl_xor_sync(0xffffffffu, v2, o);
                }
                if (lane == c) { sgx += v0; sgy += v1; sgt += v2; }
            }
        }

        // ---- store the collided pair: one contiguous run per plane and pass
        T *base = A.dst + (long long)y * L.pitch + x;
        if (act_b) {
#pragma unroll
            for (int i = 0; i < 9; ++i) Storage<T>::store2(base + i * L.plane, dk[i]);
        } else if (act_a) {
#pragma unroll
            for (int i = 0; i < 9; ++i) Storage<T>::store1(base + i * L.plane, dk[i].x);
        }
    }

    if (MODE == MODE_FIELDS) return true;
    if (__any_sync(0xffffffffu, badmax > 0x7f7ffffeu) && lane == 0) atomicOr(A.err, ERR_UNSTABLE);
    // ---- this row segment's force / torque per candidate (zero where no node is owned)
    if (lane < ncand)
        A.partial[((long long)tile * MAXC + lane) * TILE_H + (y - ty0)] = make_float4(sgx, sgy, sgt, 0.f);
    return true;
}

// Shared-memory carve-up common to both sweep kernels.
template <typename T, int W>
struct SweepSmem {
    T *stages;
    float4 *crec;
    int *cid;
    uint64_t *bars;
    __device__ __forceinline__ SweepSmem(unsigned char *raw, int warp) {
        constexpr int SW = segw_of<T>();
        constexpr size_t STAGE_BYTES = (size_t)W * STAGES * stage_elems<T>() * sizeof(T);
        constexpr size_t REC_BYTES = (size_t)W * NREC * MAXC * sizeof(float4);
        constexpr size_t ID_BYTES = (size_t)W * MAXC * sizeof(int);
        stages = reinterpret_cast<T *>(raw) + (size_t)warp * STAGES * stage_elems<T>();
        crec = reinterpret_cast<float4 *>(raw + STAGE_BYTES) + (size_t)warp * NREC * MAXC;
        cid = reinterpret_cast<int *>(raw + STAGE_BYTES + REC_BYTES) + warp * MAXC;
        bars = reinterpret_cast<uint64_t *>(raw + STAGE_BYTES + REC_BYTES + ID_BYTES) + warp * STAGES;
    }
};

// Resident warps per SM the sweep kernels are compiled for: W warps per
// block and SWEEP_SM_WARPS / W blocks per SM (registers capped at 96 per
// thread for W = 2 and 4; W = 8 holds two blocks, 16 warps).
constexpr int SWEEP_SM_WARPS = 20;

// The sweep over one lattice.  Persistent: warps take row segments
// round-robin (neighbouring warps on neighbouring segments); each warp keeps
// STAGES segments staged ahead.  W warps per block (rows in flight per
// block).
template <typename T, int MODE, bool EDGES, int W = SWEEP_WARPS, bool PS = false>
__global__ void __launch_bounds__(W * 32, SWEEP_SM_WARPS / W)
sweep_kernel(const __grid_constant__ SweepArgs<T> one)
{
    constexpr int SW = segw_of<T>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    SweepSmem<T, W> sm(smem_raw, warp);
    Ring ring;
    ring.bars = sm.bars;
    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&ring.bars[s], 1);
        mbar_fence_init();
    }
    __syncwarp();
    const Lattice &L = one.L;
    // the next step's bins start empty (nothing reads them during this sweep)
    if (one.clear)
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L.ntx * L.nty; t += gridDim.x * blockDim.x)
            one.clear[t] = 0;

    const int nitems = L.ny * L.ntx;
    const int gw = blockIdx.x * W + warp, nw = gridDim.x * W;
    // item = y * ntx + tx, advanced by nw per iteration without dividing
    const int dy_step = nw / L.ntx, dtx_step = nw - dy_step * L.ntx;
    auto advance = [&](int &yy, int &xx) {
        xx += dtx_step;
        yy += dy_step;
        if (xx >= L.ntx) { xx -= L.ntx; ++yy; }
    };
    int y = gw / L.ntx, tx = gw - (gw / L.ntx) * L.ntx;
    ring.parity = 0;
    ring.pending = 0;
    T wv = T();         // the staged segment's periodic-edge value (wrap_load)
    {
        int py = y, ptx = tx;
        for (int s = 0; s < STAGES; ++s) {
            if (gw + s * nw < nitems) {
                issue_segment<T>(one.src, L, py, ptx, sm.stages + s * stage_elems<T>(), &ring.bars[s], lane);
                wv = wrap_load<T>(one.src, L, py, ptx, lane);
                ring.pending |= 1u << s;
            }
            advance(py, ptx);
        }
    }
    // (row, segment) STAGES items ahead, for the stage being recycled
    int ay = y, atx = tx;
    for (int s = 0; s < STAGES; ++s) advance(ay, atx);

    int k = 0;
    bool timed_out = false;
    for (int item = gw; item < nitems; item += nw, ++k) {
        if (k > 0) {
            advance(y, tx);
            advance(ay, atx);
        }
        const int s = k % STAGES;
        const bool has_next = item + STAGES * nw < nitems;
        if (!sweep_segment<T, MODE, EDGES, PS>(one, y, tx, sm.stages + s * stage_elems<T>(), ring, s, has_next, one, ay, atx,
                                           sm.crec, sm.cid, wv, lane)) {
            timed_out = true;
            break;
        }
    }
    if (timed_out) {
        if (lane == 0) atomicOr(one.err, ERR_TIMEOUT);
        // let the copies this warp still has in flight land before the block
        // releases its shared memory (each wait bounded again)
        for (int s = 0; s < STAGES; ++s)
            if (ring.pending & (1u << s)) mbar_wait_bounded(&ring.bars[s], (ring.parity >> s) & 1u);
    }
}

// Position in a batched work list: item, its lattice, row and segment.
struct Cursor {
    int item, lat, y, tx;
};

// Move cursor c (at an earlier item, or c.lat = 0) forward to `item`: a
// warp's items only grow, so its lattice is found by stepping on from the
// last one (a few lattices at most per step of the work list).
template <typename T>
__device__ __forceinline__ void cursor_seek(const BatchArgs<T> &ba, Cursor &c, int item) {
    c.item = item;
    while (c.lat + 1 < ba.n && ba.item_start[c.lat + 1] <= item) ++c.lat;
    const int local = item - ba.item_start[c.lat];
    const int ntx = ba.a[c.lat].L.ntx;
    c.y = local / ntx;
    c.tx = local - c.y * ntx;
}

// The sweep over a batch of lattices (at most BATCH_LAUNCH_MAX per launch).
// Warps take the concatenated row segments round-robin, as in the
// single-lattice sweep, so that neighbouring warps stage neighbouring rows
// (DRAM page locality); each item finds its lattice by a binary search in the
// parameter space.
template <typename T, int MODE, int W = SWEEP_WARPS>
__global__ void __launch_bounds__(W * 32, SWEEP_SM_WARPS / W)
sweep_batch_kernel(const __grid_constant__ BatchArgs<T> ba)
{
    constexpr int SW = segw_of<T>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    SweepSmem<T, W> sm(smem_raw, warp);
    Ring ring;
    ring.bars = sm.bars;
    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&ring.bars[s], 1);
        mbar_fence_init();
    }
    __syncwarp();
    {
        const int ntiles = ba.tile_start[ba.n];
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
            const int lat = batch_find(ba.tile_start, ba.n, t);
            if (ba.a[lat].clear) ba.a[lat].clear[t - ba.tile_start[lat]] = 0;
        }
    }

    const int nitems = ba.item_start[ba.n];
    const int gw = blockIdx.x * W + warp, nw = gridDim.x * W;
    Cursor cur{0, 0, 0, 0}, ahead{0, 0, 0, 0};
    ring.parity = 0;
    ring.pending = 0;
    T wv = T();         // the staged segment's periodic-edge value (wrap_load)
    for (int s = 0; s < STAGES; ++s) {
        const int it = gw + s * nw;
        if (it < nitems) {
            cursor_seek(ba, ahead, it);
            issue_segment<T>(ba.a[ahead.lat].src, ba.a[ahead.lat].L, ahead.y, ahead.tx,
                             sm.stages + s * stage_elems<T>(), &ring.bars[s], lane);
            wv = wrap_load<T>(ba.a[ahead.lat].src, ba.a[ahead.lat].L, ahead.y, ahead.tx, lane);
            ring.pending |= 1u << s;
        }
    }

    int k = 0;
    bool timed_out = false;
    int last_lat = 0;
    for (int item = gw; item < nitems; item += nw, ++k) {
        const int s = k % STAGES;
        cursor_seek(ba, cur, item);
        last_lat = cur.lat;
        const int nxt = item + STAGES * nw;
        const bool has_next = nxt < nitems;
        if (has_next) cursor_seek(ba, ahead, nxt);
        const int nlat = has_next ? ahead.lat : cur.lat;
        if (!sweep_segment<T, MODE, true>(ba.a[cur.lat], cur.y, cur.tx, sm.stages + s * stage_elems<T>(), ring, s,
                                          has_next, ba.a[nlat], ahead.y, ahead.tx, sm.crec, sm.cid, wv, lane)) {
            timed_out = true;
            break;
        }
    }
    if (timed_out) {
        if (lane == 0) atomicOr(ba.a[last_lat].err, ERR_TIMEOUT);
        for (int s = 0; s < STAGES; ++s)
            if (ring.pending & (1u << s)) mbar_wait_bounded(&ring.bars[s], (ring.parity >> s) & 1u);
    }
}

// ------------------------------------------------------------ particles
struct BodyParams {
    int np;
    double gx, gy, rho_f;
    double eps_p, eps_p2, eps_w, eps_w2, xi;
};

// Map k in [0, total) of a tile-range set to its tile index, ranges in order.
__device__ __forceinline__ int range_at(const AxisTiles &a, int k) {
    const int n0 = a.hi[0] - a.lo[0] + 1;
    return k < n0 ? a.lo[0] + k : a.lo[1] + (k - n0);
}

__device__ __forceinline__ int range_len(const AxisTiles &a) {
    int n = 0;
    for (int r = 0; r < a.n; ++r) n += a.hi[r] - a.lo[r] + 1;
    return n;
}

// The particle update, per particle.  With integrate != 0:
//   1. hydrodynamic force and torque (Eqs. 18-19): the row-segment partials of
//      the tiles the particle was binned into, summed in FP64 in a fixed
//      order (lanes take fixed (tile, row) entries, then a fixed shuffle tree);
//   2. Wan-Turek repulsion (Eqs. 28-29) from the other particles (lanes stride
//      over them) and from mirror images across the walls;
//   3. symplectic Euler of Eqs. 22-24 (dt = 1), positions read from copy
//      `pin` and written to copy `pout`.
// Always, finally: binning of the particle into every tile its phi tail
// reaches (see particles_kernel for how the work is split).
// Everything one lattice's particle update needs.
struct PartArgs {
    Lattice L;
    Physics ph;
    Particles P;
    BodyParams bp;
    Bins bin_in, bin_out;       // bins the sweep used / bins for the next sweep
    const float4 *partial;
    int pin, pout;              // position copy read / written
    int integrate;
    double *force, *fcol;
    double *fsum;               // nullable: running sum of (Fx, Fy, T) over integrating steps
    int *err;
    int track = -1;             // moving frame: tracked particle, -1 (the default) when off
    double track_x = 0.0;       // its reference x
    // A strip of the lattice (L is the whole lattice): bins hold the tile rows
    // [ty_lo, ty_hi) only, local tile index (ty - ty_lo) * ntx + tx.
    int ty_lo = 0, ty_hi = 1 << 30;
    // phase 0: the whole update; 1: only the force / torque and repulsion
    // sums of this strip's bins, written to fpart (5 per particle: Fx, Fy, T,
    // repulsion x, y); 2: the rest of the update from the sums in fpart.
    int phase = 0;
    double *fpart = nullptr;
};

// v wrapped into [0, n) on a periodic axis: fmod(v, n), plus n when it is
// negative.  A position moves by less than a period per step, so within
// (-n, 2n) one subtraction or addition of n gives exactly that result (the
// difference is representable); fmod takes anything farther, and NaN.
__host__ __device__ inline double wrap_period(double v, double n) {
    if (v >= 0.0 && v < n) return v;
    if (v >= n && v < 2.0 * n) return v - n;
    if (v < 0.0 && v > -n) return v + n;
    const double w = fmod(v, n);
    return w < 0.0 ? w + n : w;
}

// Moving computational domain (Sec. 3.5): the frame's move at the end of a
// step, in columns, from the tracked particle's x at the start of that step
// (minimum image on a periodic x axis): +1 once it is one lattice unit or
// more ahead of the reference, -1 once one or more behind.
__host__ __device__ inline int frame_move(double xt, double xref, int nx, int per_x) {
    double d = xt - xref;
    if (per_x) {
        while (d >= 0.5 * nx) d -= nx;
        while (d < -0.5 * nx) d += nx;
    }
    return d >= 1.0 ? 1 : (d <= -1.0 ? -1 : 0);
}

// The particles kernel takes PART_WARPS particles per block, in three phases:
// (A) each particle's warp sums its force partials and finds its Wan-Turek
// contacts; (B) one lane per particle does the scalar FP64 work (walls,
// rigid-body update, frame move, velocity splits, tile ranges); (C) each warp
// bins its particle for the next sweep.  The FP64 pipe is narrow on this part
// and charges per warp instruction whatever the mask, so one warp serving the
// block's particles in (B) costs a PART_WARPS-th of every warp doing its own.
constexpr int PART_WARPS = 8;

struct PartShared {
    double fx, fy, tq, cx, cy;      // (A) hydrodynamic force, torque; repulsion
    double nX, nY;                  // (B) position for the next step
    float4 rb;                      // (B) record: r and the velocities' FP32 hi parts
    float rlx, rly, rlz;            // (B) the velocities' FP32 lo parts
    AxisTiles ax, ay;               // (B) the tiles the particle's reach covers
};

// The position copies of a step without indexing the parameter arrays.
struct PartCopies {
    const double *xin, *yin;
    const float *xfin, *yfin;
    double *xout, *yout;
    float *xfout, *yfout;
    __device__ __forceinline__ explicit PartCopies(const PartArgs &A) {
        const Particles &P = A.P;
        xin = A.pin ? P.x[1] : P.x[0]; yin = A.pin ? P.y[1] : P.y[0];
        xfin = A.pin ? P.xf[1] : P.xf[0]; yfin = A.pin ? P.yf[1] : P.yf[0];
        xout = A.pout ? P.x[1] : P.x[0]; yout = A.pout ? P.y[1] : P.y[0];
        xfout = A.pout ? P.xf[1] : P.xf[0]; yfout = A.pout ? P.yf[1] : P.yf[0];
    }
};

// (A) Hydrodynamic force and torque (Eqs. 18-19) from the sweep's partials,
// and the particle-particle repulsion (Eq. 28), summed over the warp.  Both
// sums start from the particle's tile entries, which each lane loads once
// (entry k = lane + 32 q in register q); the first requests of the repulsion
// search (its first tile's count and first ids) go out before the force sum,
// so that the two chains of dependent loads overlap.
constexpr int PSLOT_REGS = MAXT / 32;   // tile entries per lane
static_assert(MAXT % 32 == 0 && MAXC >= 4, "tile entries are spread over whole warps");
constexpr int CONTACT_PREFETCH = 4;     // ids of the first tile requested early

__device__ __forceinline__ void particle_forces(const PartArgs &A, int p, int lane, PartShared &sh) {
    const Lattice &L = A.L;
    const Particles &P = A.P;
    const BodyParams &bp = A.bp;
    const Bins &bin_in = A.bin_in;
    const float4 *__restrict__ partial = A.partial;
    const PartCopies pc(A);
    const double *xin = pc.xin, *yin = pc.yin;
    const float *xfin = pc.xfin, *yfin = pc.yfin;
    const double X = xin[p], Y = yin[p], r = P.r[p];

    const int nk = bin_in.npslot[p];
    int tsl[PSLOT_REGS];
#pragma unroll
    for (int q = 0; q < PSLOT_REGS; ++q) {
        const int k = lane + 32 * q;
        tsl[q] = k < nk ? bin_in.pslot[(long long)p * MAXT + k] : -1;
    }
    // the repulsion search's first tile: its count and first ids (slots of
    // the tile, in bounds; used only below the count)
    const int t0 = tsl[0] >= 0 ? tsl[0] / MAXC : -1;
    int cnt0 = 0, jpre[CONTACT_PREFETCH];
    if (t0 >= 0) {
        cnt0 = bin_in.count[t0];
#pragma unroll
        for (int s = 0; s < CONTACT_PREFETCH; ++s) jpre[s] = bin_in.ids[t0 * MAXC + s];
    } else {
#pragma unroll
        for (int s = 0; s < CONTACT_PREFETCH; ++s) jpre[s] = 0;
    }

    // ---- 1. hydrodynamic force and torque: lane l adds entries e = l, l + 32,
    // ... (tile entry e / TILE_H, row e % TILE_H) in that order
    double fx = 0.0, fy = 0.0, tq = 0.0;
    const int ne = nk * TILE_H;
#pragma unroll 2
    for (int base = 0; base < ne; base += 32) {
        const int e = base + lane;
        const int k = e / TILE_H, row = e - k * TILE_H;
        // entry k sits in lane k % 32, register k / 32 = base / (32 TILE_H)
        // (the same for the whole warp in one iteration)
        const int q = base / (32 * TILE_H);
        int src = tsl[0];
#pragma unroll
        for (int qq = 1; qq < PSLOT_REGS; ++qq)
            if (q == qq) src = tsl[qq];
        const int ts = __shfl_sync(0xffffffffu, src, k & 31);
        if (e >= ne || ts < 0) continue;
        const int ty = (ts / MAXC) / L.ntx + A.ty_lo;
        if (ty * TILE_H + row >= L.ny) continue;
        const float4 v = partial[(long long)ts * TILE_H + row];
        fx += (double)v.x; fy += (double)v.y; tq += (double)v.z;
    }
    // ---- 2. particle-particle repulsion.  A pair within r_i + r_j + xi
    // shares the tile holding the middle of the gap between the surfaces
    // (that point lies inside both binning reaches), so each lane takes
    // some of this particle's tiles and counts a pair only in that tile;
    // within a tile the pairs are added in increasing partner id.
    double cx = 0.0, cy = 0.0;
    const float xf = xfin[p], yf = yfin[p], rf = (float)r;
#pragma unroll
    for (int q = 0; q < PSLOT_REGS; ++q) {
        if (lane + 32 * q >= nk) break;
        const int ts = tsl[q];
        if (ts < 0) continue;
        const int t = ts / MAXC;
        int n = q == 0 ? cnt0 : bin_in.count[t];
        n = n > MAXC ? MAXC : n;
        uint32_t contact = 0;
        for (int sl = 0; sl < n; ++sl) {
            int j;
            if (q == 0 && sl < CONTACT_PREFETCH)
                j = sl == 0 ? jpre[0] : (sl == 1 ? jpre[1] : (sl == 2 ? jpre[2] : jpre[3]));
            else
                j = bin_in.ids[t * MAXC + sl];
            if (j == p) continue;
            float dxf = xf - xfin[j], dyf = yf - yfin[j];
            if (L.per_x) { if (dxf >= 0.5f * L.nx) dxf -= L.nx; else if (dxf < -0.5f * L.nx) dxf += L.nx; }
            if (L.per_y) { if (dyf >= 0.5f * L.ny) dyf -= L.ny; else if (dyf < -0.5f * L.ny) dyf += L.ny; }
            const float lim = rf + (float)P.r[j] + (float)bp.xi + 0.05f;
            if (dxf * dxf + dyf * dyf > lim * lim) continue;
            double dx = X - xin[j], dy = Y - yin[j];
            if (L.per_x) { while (dx >= 0.5 * L.nx) dx -= L.nx; while (dx < -0.5 * L.nx) dx += L.nx; }
            if (L.per_y) { while (dy >= 0.5 * L.ny) dy -= L.ny; while (dy < -0.5 * L.ny) dy += L.ny; }
            // the middle of the gap between the two surfaces, at distance
            // (d + r - r_j) / 2 from this centre toward the partner
            const double dd = sqrt(dx * dx + dy * dy);
            const double f = dd > 0.0 ? 0.5 * (dd + r - P.r[j]) / dd : 0.0;
            double mx = X - f * dx, my = Y - f * dy;
            if (L.per_x) mx = wrap_period(mx, (double)L.nx);
            if (L.per_y) my = wrap_period(my, (double)L.ny);
            int mxi = (int)floor(mx), myi = (int)floor(my);
            mxi = mxi < 0 ? 0 : (mxi > L.nx - 1 ? L.nx - 1 : mxi);
            myi = myi < 0 ? 0 : (myi > L.ny - 1 ? L.ny - 1 : myi);
            if ((myi / TILE_H) * L.ntx + mxi / TILE_W == t + A.ty_lo * L.ntx) contact |= 1u << sl;
        }
        while (contact) {                         // increasing partner id
            int sel = -1, jmin = 0x7fffffff;
            for (uint32_t m = contact; m; m &= m - 1) {
                const int sl = __ffs(m) - 1, j = bin_in.ids[t * MAXC + sl];
                if (j < jmin) { jmin = j; sel = sl; }
            }
            contact &= ~(1u << sel);
            double dx = X - xin[jmin], dy = Y - yin[jmin];
            if (L.per_x) { while (dx >= 0.5 * L.nx) dx -= L.nx; while (dx < -0.5 * L.nx) dx += L.nx; }
            if (L.per_y) { while (dy >= 0.5 * L.ny) dy -= L.ny; while (dy < -0.5 * L.ny) dy += L.ny; }
            const double d = sqrt(dx * dx + dy * dy), rr = r + P.r[jmin];
            double sc = 0.0;
            if (d <= rr) sc = (rr - d) / bp.eps_p2;
            else if (d <= rr + bp.xi) sc = (rr + bp.xi - d) * (rr + bp.xi - d) / bp.eps_p;
            cx += sc * dx;
            cy += sc * dy;
        }
    }
    // (the repulsion sums, zero unless some lane found a contact, are
    // reduced only when one did)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        tq += __shfl_xor_sync(0xffffffffu, tq, o);
    }
    if (__any_sync(0xffffffffu, cx != 0.0 || cy != 0.0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cx += __shfl_xor_sync(0xffffffffu, cx, o);
            cy += __shfl_xor_sync(0xffffffffu, cy, o);
        }
    }
    if (lane == 0) {
        sh.fx = fx; sh.fy = fy; sh.tq = tq; sh.cx = cx; sh.cy = cy;
    }
}

// The particle state (B) reads, loaded at the start of the kernel so that
// its latency passes while the warps sum their forces.
struct PartState {
    double X, Y, r, ux, uy, om, rho_s, theta;
    int fixed;
};

__device__ __forceinline__ PartState load_state(const PartArgs &A, int p) {
    const Particles &P = A.P;
    const PartCopies pc(A);
    PartState st;
    st.X = pc.xin[p]; st.Y = pc.yin[p]; st.r = P.r[p];
    st.ux = P.ux[p]; st.uy = P.uy[p]; st.om = P.omega[p];
    st.rho_s = P.rho_s[p]; st.theta = P.theta[p]; st.fixed = P.fixed[p];
    return st;
}

// (B) One thread per particle: wall repulsion (Eq. 29), the rigid-body
// update (Eqs. 22-24), the frame move, the position copies for the next step,
// and what the binning needs (velocity splits, the tiles the reach covers).
__device__ __forceinline__ void particle_update(const PartArgs &A, int p, PartShared &sh, const PartState &st) {
    const Lattice &L = A.L;
    const Physics &ph = A.ph;
    const Particles &P = A.P;
    const BodyParams &bp = A.bp;
    const PartCopies pc(A);
    const double X = st.X, Y = st.Y, r = st.r;
    double nX = X, nY = Y;
    double ux = st.ux, uy = st.uy, om = st.om;

    if (A.integrate) {
        const double fx = sh.fx, fy = sh.fy, tq = sh.tq;
        double cx = sh.cx, cy = sh.cy;
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
            double sc = 0.0;
            if (d <= rr) sc = (rr - d) / bp.eps_w2;
            else if (d <= rr + bp.xi) sc = (rr + bp.xi - d) * (rr + bp.xi - d) / bp.eps_w;
            cx += sc * dx;
            cy += sc * dy;
        }
        // ---- 3. rigid-body update
        if (!st.fixed) {
            // two FP64 divisions instead of four: the buoyancy-reduced weight
            // (1 - rho_f / rho_s) m g is (rho_s - rho_f) pi r^2 g
            const double area = 3.14159265358979323846 * r * r;
            const double m = st.rho_s * area;
            const double im = 1.0 / m, iI = 1.0 / (0.5 * m * r * r);
            const double wgt = (st.rho_s - bp.rho_f) * area;        // buoyancy-reduced weight / g
            ux += (fx + cx + wgt * bp.gx) * im;
            uy += (fy + cy + wgt * bp.gy) * im;
            om += tq * iI;
            nX = X + ux;
            nY = Y + uy;
            if (L.per_x) nX = wrap_period(nX, (double)L.nx);
            if (L.per_y) nY = wrap_period(nY, (double)L.ny);
            P.ux[p] = ux; P.uy[p] = uy; P.omega[p] = om;
            P.theta[p] = st.theta + om;
        }
        A.force[3 * p] = fx; A.force[3 * p + 1] = fy; A.force[3 * p + 2] = tq;
        A.fcol[2 * p] = cx; A.fcol[2 * p + 1] = cy;
        if (A.fsum) {
            A.fsum[3 * p] += fx; A.fsum[3 * p + 1] += fy; A.fsum[3 * p + 2] += tq;
        }
        if (A.track >= 0) {
            // the frame moves with the tracked particle: every particle, fixed
            // ones included, shifts by the same whole number of columns
            const int s = frame_move(pc.xin[A.track], A.track_x, L.nx, L.per_x);
            if (s) {
                nX -= (double)s;
                if (L.per_x) nX = wrap_period(nX, (double)L.nx);
            }
        }
    }
    pc.xout[p] = nX; pc.yout[p] = nY;
    pc.xfout[p] = (float)nX; pc.yfout[p] = (float)nY;

    // velocities as FP32 hi + lo: the sweep forms u_s - u*, a small difference
    const float uxh = (float)ux, uyh = (float)uy, omh = (float)om;
    sh.nX = nX; sh.nY = nY;
    sh.rb = make_float4((float)r, uxh, uyh, omh);
    sh.rlx = (float)(ux - (double)uxh); sh.rly = (float)(uy - (double)uyh); sh.rlz = (float)(om - (double)omh);
    const double R = r + ph.cut_d;
    sh.ax = axis_tiles(nX, R, L.nx, TILE_W, L.ntx, L.per_x);
    sh.ay = axis_tiles(nY, R, L.ny, TILE_H, L.nty, L.per_y);
}

// (C) Binning of the particle into every tile its reach covers (lanes take
// the tiles in a fixed order), with the record the sweep reads: the centre
// relative to the tile origin (minimum image about the tile centre) as FP32
// hi + lo, radius and velocities.
__device__ __forceinline__ void particle_bin(const PartArgs &A, int p, int lane, const PartShared &sh) {
    const Lattice &L = A.L;
    const Bins &bin_out = A.bin_out;
    const double nX = sh.nX, nY = sh.nY;
    const AxisTiles ax = sh.ax, ay = sh.ay;
    const float4 rb = sh.rb;
    const float rlx = sh.rlx, rly = sh.rly, rlz = sh.rlz;
    const int NX = range_len(ax), NY = range_len(ay);
    int total = NX * NY;
    if (total > MAXT) {                      // ruled out at create; kept as a guard
        if (lane == 0) atomicOr(A.err, ERR_OVERFLOW);
        total = MAXT;
    }
    for (int k = lane; k < total; k += 32) {
        const int ty = range_at(ay, k / NX), tx = range_at(ax, k - (k / NX) * NX);
        int entry = -1;
        if (ty < A.ty_lo || ty >= A.ty_hi) {       // another strip's tile
            bin_out.pslot[(long long)p * MAXT + k] = entry;
            continue;
        }
        const int t = (ty - A.ty_lo) * L.ntx + tx;
        const int s = atomicAdd(&bin_out.count[t], 1);
        if (s < MAXC) {
            double cx = nX - (double)(tx * TILE_W), cy = nY - (double)(ty * TILE_H);
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
            entry = t * MAXC + s;
            bin_out.ids[entry] = p;
            bin_out.rec[NREC * (long long)entry] = make_float4(cxh, (float)(cx - (double)cxh), cyh, (float)(cy - (double)cyh));
            bin_out.rec[NREC * (long long)entry + 1] = rb;
            // the centre's whole-cell offsets from the tile origin (the PS sweep's table index)
            const int fxi = (int)floor(cx), fyi = (int)floor(cy);
            bin_out.rec[NREC * (long long)entry + 2] =
                make_float4(rlx, rly, rlz, __int_as_float((fxi & 0xffff) | (int)((unsigned)fyi << 16)));
        } else {
            atomicOr(A.err, ERR_OVERFLOW);
        }
        bin_out.pslot[(long long)p * MAXT + k] = entry;
    }
    if (lane == 0) bin_out.npslot[p] = total;
}

// PART_WARPS particles per block of one lattice (BATCH = false) or of every
// lattice of a batch (BATCH = true; bi.item_start holds each lattice's first
// particle).  Launch with PART_WARPS * 32 threads and ceil(particles /
// PART_WARPS) blocks.
template <bool BATCH>
__global__ void __launch_bounds__(PART_WARPS * 32)
particles_kernel(const __grid_constant__ PartArgs one, const PartArgs *__restrict__ many, BatchIndex bi) {
    __shared__ PartShared sh[PART_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int total = BATCH ? bi.item_start[bi.n] : one.bp.np;
    // the arguments and index of item g (a particle), or null past the end
    auto locate = [&](int g, int &p) -> const PartArgs * {
        if (g >= total) return nullptr;
        if constexpr (BATCH) {
            const int lat = batch_find(bi.item_start, bi.n, g);
            p = g - bi.item_start[lat];
            return &many[lat];
        } else {
            p = g;
            return &one;
        }
    };
    int p = 0;
    const PartArgs *A = locate(blockIdx.x * PART_WARPS + w, p);
    const int phase = BATCH ? 0 : one.phase;       // (uniform over the launch)
    // (B)'s lanes: their particle and its state, requested now
    int q = 0;
    const PartArgs *B = nullptr;
    PartState st{};
    if (phase != 1 && w == 0 && lane < PART_WARPS) {
        B = locate(blockIdx.x * PART_WARPS + lane, q);
        if (B) st = load_state(*B, q);
    }
    if (A && A->integrate && phase != 2) particle_forces(*A, p, lane, sh[w]);
    if (phase == 1) {
        if (A && A->integrate && lane == 0) {
            double *o = A->fpart + 5 * (long long)p;
            o[0] = sh[w].fx; o[1] = sh[w].fy; o[2] = sh[w].tq; o[3] = sh[w].cx; o[4] = sh[w].cy;
        }
        return;
    }
    if (phase == 2 && A && lane == 0) {
        const double *o = A->fpart + 5 * (long long)p;
        sh[w].fx = o[0]; sh[w].fy = o[1]; sh[w].tq = o[2]; sh[w].cx = o[3]; sh[w].cy = o[4];
    }
    __syncthreads();
    if (B) particle_update(*B, q, sh[lane], st);
    __syncthreads();
    if (A) particle_bin(*A, p, lane, sh[w]);
}

// ------------------------------------------------------------ conversions
// e_i of direction i given at run time (the conversion kernels index by a
// computed direction).
__device__ __forceinline__ float ref_e_of(const Lattice &L, int i) {
    float v = L.ref_e[0];
#pragma unroll
    for (int j = 1; j < 9; ++j)
        if (i == j) v = L.ref_e[j];
    return v;
}

// Populations <-> FP64 f_i (dense 9 x ny x nx) for checkpoints.
template <typename T>
__global__ void export_kernel(const T *__restrict__ src, Lattice L, double *__restrict__ out) {
    const long long n = (long long)L.nx * L.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 9 * n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / n);
        const long long r = k - i * n;
        const int y = (int)(r / L.nx), x = (int)(r - (long long)y * L.nx);
        const double v = (double)Storage<T>::load1(src + i * L.plane + (long long)y * L.pitch + x);
        out[k] = (std::is_same<T, float>::value ? v : v * (double)L.ref_q + (double)ref_e_of(L, i)) + (double)wof(i);
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
        const double dv = in[k] - w[i];
        Storage<T>::store1(dst + i * L.plane + (long long)y * L.pitch + x,
                           std::is_same<T, float>::value ? (float)dv
                                                         : (float)((dv - (double)ref_e_of(L, i)) * (double)L.ref_iq));
    }
}

// Uniform initial state f^eq(rho0, u0) written as deviations on every node.
// PS-LBM (Sec. 2.2): the covered area of every cell about each particle
// (B = eps_s, Eq. 8), once per step after the particle update, for the next
// sweep to look up.  Particle p's table holds the (2K+1)^2 cells about
// (floor X, floor Y), row-major; the cell at offset (i, j) is the node
// (floor X + i, floor Y + j).  The same decisions as the sweep's: 0 beyond
// the reach r + cut, 1 once every corner is inside.  One block per particle
// walks its table; the particle's fractional centre is formed once in FP64
// and shared as FP32 hi + lo.  The cells the circle crosses (about one in
// eight, scattered over every warp) are gathered first and then summed by
// whole warps; cells past the list's capacity (only for very large discs)
// are summed where they are found.
constexpr int COVER_BX = 32, COVER_BY = 8, COVER_RING = 2048;

static __global__ void __launch_bounds__(COVER_BX * COVER_BY)
cover_kernel(float *__restrict__ cover, const double *__restrict__ xs, const double *__restrict__ ys,
             const double *__restrict__ rs, int np, Physics ph) {
    __shared__ int ring[COVER_RING];
    __shared__ int nring;
    __shared__ float frac[5];               // x - floor x (hi, lo), y - floor y (hi, lo), r
    const int tid = threadIdx.y * COVER_BX + threadIdx.x;
    const int K = ph.ck, S = 2 * K + 1;
    for (int p = blockIdx.x; p < np; p += gridDim.x) {
        if (tid == 0) {
            nring = 0;
            const double X = xs[p], Y = ys[p];
            const double fx = X - floor(X), fy = Y - floor(Y);
            frac[0] = (float)fx;
            frac[1] = (float)(fx - (double)frac[0]);
            frac[2] = (float)fy;
            frac[3] = (float)(fy - (double)frac[2]);
            frac[4] = (float)rs[p];
        }
        __syncthreads();
        const float rf = frac[4], Rf = rf + ph.cut;
        float *tab = cover + (long long)p * S * S;
        for (int iy = threadIdx.y; iy < S; iy += COVER_BY) {
            const float dy = ((float)(iy - K) - frac[2]) - frac[3];
            for (int ix = threadIdx.x; ix < S; ix += COVER_BX) {
                const float dx = ((float)(ix - K) - frac[0]) - frac[1];
                const float d2 = dx * dx + dy * dy;
                float v = 0.f;
                bool crossed = false;
                if (d2 <= Rf * Rf) {
                    const float l = rf - sqrtf(d2);
                    if (l >= ph.cut) v = 1.0f;
                    else crossed = l >= -ph.cut;
                }
                if (crossed) {
                    const int slot = atomicAdd(&nring, 1);
                    if (slot < COVER_RING) ring[slot] = iy * S + ix;
                    else tab[iy * S + ix] = cell_cover(dx, dy, rf);
                } else {
                    tab[iy * S + ix] = v;
                }
            }
        }
        __syncthreads();
        const int nr = nring < COVER_RING ? nring : COVER_RING;
        for (int k = tid; k < nr; k += COVER_BX * COVER_BY) {
            const int j = ring[k], cy = j / S, cx = j - cy * S;
            const float dx = ((float)(cx - K) - frac[0]) - frac[1], dy = ((float)(cy - K) - frac[2]) - frac[3];
            tab[j] = cell_cover(dx, dy, rf);
        }
        __syncthreads();
    }
}

// Moving computational domain (Sec. 3.5): when the frame moves by s columns
// (decided from the tracked particle's x at the start of the step that just
// ran, as the particle update decided it), column x of every population
// plane takes the stored values of column x + s: rolled on a periodic x
// axis, otherwise clamped, so the entering column repeats its neighbour.
// The move is in place, one row of one plane at a time through shared
// memory (nx elements); block 0 adds s to the frame offset.
template <typename T>
__global__ void frame_shift_kernel(T *__restrict__ buf, Lattice L, const double *__restrict__ xt, int track,
                                   double track_x, long long *__restrict__ offset) {
    extern __shared__ __align__(16) unsigned char frame_row[];
    T *row = reinterpret_cast<T *>(frame_row);
    const int s = frame_move(xt[track], track_x, L.nx, L.per_x);
    if (s == 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *offset += s;
    for (int y = blockIdx.x; y < L.ny; y += gridDim.x) {
        for (int i = 0; i < 9; ++i) {
            T *line = buf + (long long)i * L.plane + (long long)y * L.pitch;
            for (int x = threadIdx.x; x < L.nx; x += blockDim.x) row[x] = line[x];
            __syncthreads();
            for (int x = threadIdx.x; x < L.nx; x += blockDim.x) {
                int src = x + s;
                if (L.per_x) src = src < 0 ? src + L.nx : (src >= L.nx ? src - L.nx : src);
                else src = src < 0 ? 0 : (src > L.nx - 1 ? L.nx - 1 : src);
                line[x] = row[src];
            }
            __syncthreads();
        }
    }
}

template <typename T>
__global__ void init_kernel(T *__restrict__ dst, Lattice L, float drho, float ux, float uy) {
    const long long n = (long long)L.nx * L.ny;
    float e[9];
    eq_dev9(drho, 1.0f + drho, ux, uy, e);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 9 * n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / n);
        const long long r = k - i * n;
        const int y = (int)(r / L.nx), x = (int)(r - (long long)y * L.nx);
        float v = e[0];
#pragma unroll
        for (int j = 1; j < 9; ++j)
            if (i == j) v = e[j];
        // (16-bit storage: the initial state is the reference state itself, s_i = 0)
        Storage<T>::store1(dst + i * L.plane + (long long)y * L.pitch + x, std::is_same<T, float>::value ? v : 0.0f);
    }
}

}  // namespace dilbm
