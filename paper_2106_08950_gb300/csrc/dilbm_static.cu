// dilbm_step_static: one DI-LBM time step on caller-owned device buffers that
// allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need a
// step: a solver that owns a fixed memory pool and forbids further device
// allocations, a code path that must not call cudaMalloc because it would
// synchronise the device in the middle of a stream-ordered pipeline, or a
// host that has budgeted every byte of the GPU up front.  For them this entry
// point runs the same kernels as dilbm_step (sweep_kernel, particles_kernel)
// with every piece of scratch memory (tile bins, force partials, the particle
// state in structure-of-arrays form, the error word) taken from one
// file-scope static device array of fixed size, declared below.  The caller
// passes the populations, the particles and the force output.
#include "dilbm.h"
#include "dilbm_kernels.cuh"

#include <cmath>
#include <string>

using namespace dilbm;

namespace {

// Limits of the static scratch (also stated in include/dilbm.h).
constexpr int S_MAX_TILES = DILBM_STATIC_MAX_TILES;       // 128 x 8-node tiles
constexpr int S_MAX_PARTICLES = DILBM_STATIC_MAX_PARTICLES;
// The caller's population layout is the kernels' own: the header's offset is
// the readable guard the bulk copies rely on, and its pitch is the kernels'.
static_assert(GUARD == DILBM_STATIC_POP_OFFSET, "DILBM_STATIC_POP_OFFSET must equal the sweep's guard");
static_assert(DILBM_STATIC_PITCH(1) == 32 && DILBM_STATIC_PITCH(33) == 64, "pitch: nx rounded up to 32");

// Byte offsets of the scratch regions (each 256-byte aligned).
constexpr size_t align256(size_t n) { return (n + 255) / 256 * 256; }
constexpr size_t OFF_COUNT = 0;                                                    // int [2][tiles]
constexpr size_t OFF_IDS = OFF_COUNT + align256(2 * sizeof(int) * S_MAX_TILES);    // int [2][tiles*MAXC]
constexpr size_t OFF_REC = OFF_IDS + align256(2 * sizeof(int) * S_MAX_TILES * MAXC);
constexpr size_t OFF_PSLOT = OFF_REC + align256(2 * sizeof(float4) * S_MAX_TILES * MAXC * NREC);
constexpr size_t OFF_NPSLOT = OFF_PSLOT + align256(2 * sizeof(int) * S_MAX_PARTICLES * MAXT);
constexpr size_t OFF_PARTIAL = OFF_NPSLOT + align256(2 * sizeof(int) * S_MAX_PARTICLES);
constexpr size_t OFF_PD = OFF_PARTIAL + align256(sizeof(float4) * S_MAX_TILES * MAXC * TILE_H);
constexpr size_t OFF_PF = OFF_PD + align256(10 * sizeof(double) * S_MAX_PARTICLES);
constexpr size_t OFF_FIXED = OFF_PF + align256(4 * sizeof(float) * S_MAX_PARTICLES);
constexpr size_t OFF_FCOL = OFF_FIXED + align256(sizeof(int) * S_MAX_PARTICLES);
constexpr size_t OFF_ERR = OFF_FCOL + align256(2 * sizeof(double) * S_MAX_PARTICLES);
constexpr size_t SCRATCH_BYTES = OFF_ERR + 256;

// The scratch itself.  Every GPU that loads this library holds it until the
// process exits; every call shares it, and it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_static_scratch[SCRATCH_BYTES];

}  // namespace

namespace dilbm {
int set_last_error(int code, const std::string &msg);   // dilbm.cu: the message dilbm_last_error() returns
}

namespace {

int sfail(int code, const std::string &msg) { return dilbm::set_last_error(code, msg); }

int scuda(cudaError_t e, const char *what) {
    return sfail(DILBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define S_CUDA(call)                                     \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return scuda(e_, #call);  \
    } while (0)

// Device address of the scratch array, looked up once per device with that
// device current.  In host code the array's name is only a host-side stand-in.
unsigned char *g_scratch_ptr[64] = {};

int scratch_address(unsigned char **out) {
    int dev = 0;
    S_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return sfail(DILBM_ERR_INVALID_ARG, "device ordinal out of range");
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        S_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return DILBM_OK;
}

// dilbm_particle (array of structures, device) <-> the kernels' structure of
// arrays.  The particles live in device memory, so they are checked here, with
// the same rules dilbm_create applies on the host: centre inside the lattice,
// finite positive radius and density, finite velocities and angle, and a phi
// tail that reaches at most MAXT tiles.  A bad particle sets ERR_BADPARTICLE,
// and the host reads the error word before it launches anything else, so the
// binning's minimum-image loops never see an out-of-range or non-finite centre.
__global__ void particles_in_kernel(const dilbm_particle *__restrict__ in, Particles P, int np, int nx, int ny,
                                    int per_x, int per_y, double cut_d, int *__restrict__ err) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const dilbm_particle q = in[p];
    const bool inx = per_x ? (q.x >= 0.0 && q.x < nx) : (q.x >= 0.0 && q.x <= nx - 1);
    const bool iny = per_y ? (q.y >= 0.0 && q.y < ny) : (q.y >= 0.0 && q.y <= ny - 1);
    const bool finite = isfinite(q.r) && isfinite(q.rho_s) && isfinite(q.ux) && isfinite(q.uy) &&
                        isfinite(q.omega) && isfinite(q.theta);
    bool ok = inx && iny && finite && q.r > 0.0 && q.rho_s > 0.0;
    if (ok) {
        const double R = q.r + cut_d;
        const double tx = ceil((2.0 * R + 2.0) / TILE_W) + 1.0, ty = ceil((2.0 * R + 2.0) / TILE_H) + 1.0;
        ok = tx * ty <= (double)MAXT;
    }
    if (!ok) atomicOr(err, ERR_BADPARTICLE);
    P.x[0][p] = q.x; P.y[0][p] = q.y; P.x[1][p] = q.x; P.y[1][p] = q.y;
    P.r[p] = q.r; P.ux[p] = q.ux; P.uy[p] = q.uy; P.omega[p] = q.omega; P.theta[p] = q.theta;
    P.rho_s[p] = q.rho_s; P.fixed[p] = q.fixed ? 1 : 0;
    P.xf[0][p] = (float)q.x; P.yf[0][p] = (float)q.y;
}

__global__ void particles_out_kernel(dilbm_particle *__restrict__ out, Particles P, int np) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    dilbm_particle q = out[p];
    q.x = P.x[1][p]; q.y = P.y[1][p];
    q.ux = P.ux[p]; q.uy = P.uy[p]; q.omega = P.omega[p]; q.theta = P.theta[p];
    out[p] = q;
}

}  // namespace

extern "C" int dilbm_step_static(const dilbm_grid *g, double tau, double interface_width, const float *f_in,
                                 float *f_out, dilbm_particle *particles, int np, double *force, void *cuda_stream) {
    // ---- arguments (host only; nothing is launched before they pass)
    if (!g || !f_in || !f_out || f_in == f_out || (np > 0 && (!particles || !force)) || np < 0)
        return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: NULL or aliased buffer, or np < 0");
    if (g->storage != DILBM_FP32) return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: FP32 storage only");
    if (g->nx < 3 || g->ny < 3 || !(tau > 0.5) || !std::isfinite(tau) || !(interface_width > 0.0) ||
        !std::isfinite(interface_width))
        return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: nx, ny >= 3, tau > 0.5, interface width > 0");
    const dilbm_side *sides[4] = {&g->west, &g->east, &g->south, &g->north};
    for (int k = 0; k < 4; ++k)
        if (sides[k]->kind < DILBM_SIDE_PERIODIC || sides[k]->kind > DILBM_SIDE_PRESSURE ||
            (sides[k]->kind == DILBM_SIDE_PRESSURE && !(sides[k]->rho > 0.0)))
            return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: bad side");
    if ((g->west.kind == DILBM_SIDE_PERIODIC) != (g->east.kind == DILBM_SIDE_PERIODIC) ||
        (g->south.kind == DILBM_SIDE_PERIODIC) != (g->north.kind == DILBM_SIDE_PERIODIC))
        return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: an axis must be periodic on both sides or neither");
    if (g->force_model != DILBM_FORCE_EQ18 && g->force_model != DILBM_FORCE_MOMENTUM)
        return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: unknown force model");
    if (g->method != DILBM_METHOD_DI) return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: DI-LBM only");
    if (!(g->rho_f > 0.0)) return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: rho_f must be > 0");
    for (int k = 0; k < 5; ++k)
        if (!(g->wan_turek[k] > 0.0)) return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: Wan-Turek parameters must be > 0");

    Lattice L{};
    L.nx = g->nx;
    L.ny = g->ny;
    L.pitch = DILBM_STATIC_PITCH(g->nx);
    L.plane = (long long)L.pitch * L.ny;
    L.ntx = (L.nx + TILE_W - 1) / TILE_W;
    L.nty = (L.ny + TILE_H - 1) / TILE_H;
    const long long ntiles = (long long)L.ntx * L.nty;
    if (ntiles > S_MAX_TILES)
        return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: the lattice needs " + std::to_string(ntiles) +
                                                " tiles of 128 x 8 nodes; the static scratch holds " +
                                                std::to_string(S_MAX_TILES));
    if (np > S_MAX_PARTICLES)
        return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: " + std::to_string(np) +
                                                " particles; the static scratch holds " +
                                                std::to_string(S_MAX_PARTICLES));
    L.per_x = g->west.kind == DILBM_SIDE_PERIODIC;
    L.per_y = g->south.kind == DILBM_SIDE_PERIODIC;
    L.wrap_x = L.per_x;            // radii are on the device: every node takes its own minimum image
    L.wrap_y = L.per_y;
    for (int k = 0; k < 4; ++k) {
        L.side_kind[k] = sides[k]->kind;
        L.side_ux[k] = (float)sides[k]->ux;
        L.side_uy[k] = (float)sides[k]->uy;
        L.side_drho[k] = (float)(sides[k]->rho - 1.0);
    }
    Physics ph{};
    ph.omega = (float)(1.0 / tau);
    ph.kf = (float)(1.0 - 0.5 / tau);
    ph.kforce = g->force_model == DILBM_FORCE_EQ18 ? ph.kf : 1.0f;
    ph.phi_k2 = (float)(-4.0 / (interface_width * std::log(2.0)));
    ph.cut_d = PHI_CUT_WIDTHS * interface_width;
    ph.cut = (float)ph.cut_d;
    BodyParams bp{};
    bp.np = np;
    bp.gx = g->gravity[0];
    bp.gy = g->gravity[1];
    bp.rho_f = g->rho_f;
    bp.eps_p = g->wan_turek[0];
    bp.eps_p2 = g->wan_turek[1];
    bp.eps_w = g->wan_turek[2];
    bp.eps_w2 = g->wan_turek[3];
    bp.xi = g->wan_turek[4];

    // ---- the scratch regions
    unsigned char *s = nullptr;
    int rc = scratch_address(&s);
    if (rc) return rc;
    Bins bins[2]{};
    for (int b = 0; b < 2; ++b) {
        bins[b].count = reinterpret_cast<int *>(s + OFF_COUNT) + b * S_MAX_TILES;
        bins[b].ids = reinterpret_cast<int *>(s + OFF_IDS) + (size_t)b * S_MAX_TILES * MAXC;
        bins[b].rec = reinterpret_cast<float4 *>(s + OFF_REC) + (size_t)b * S_MAX_TILES * MAXC * NREC;
        bins[b].pslot = reinterpret_cast<int *>(s + OFF_PSLOT) + (size_t)b * S_MAX_PARTICLES * MAXT;
        bins[b].npslot = reinterpret_cast<int *>(s + OFF_NPSLOT) + b * S_MAX_PARTICLES;
    }
    float4 *partial = reinterpret_cast<float4 *>(s + OFF_PARTIAL);
    double *pd = reinterpret_cast<double *>(s + OFF_PD);
    float *pf = reinterpret_cast<float *>(s + OFF_PF);
    const int M = S_MAX_PARTICLES;
    Particles P{};
    P.x[0] = pd; P.x[1] = pd + M; P.y[0] = pd + 2 * M; P.y[1] = pd + 3 * M;
    P.r = pd + 4 * M; P.ux = pd + 5 * M; P.uy = pd + 6 * M; P.omega = pd + 7 * M;
    P.theta = pd + 8 * M; P.rho_s = pd + 9 * M;
    P.xf[0] = pf; P.xf[1] = pf + M; P.yf[0] = pf + 2 * M; P.yf[1] = pf + 3 * M;
    P.fixed = reinterpret_cast<int *>(s + OFF_FIXED);
    double *fcol = reinterpret_cast<double *>(s + OFF_FCOL);
    int *err = reinterpret_cast<int *>(s + OFF_ERR);

    cudaStream_t st = (cudaStream_t)cuda_stream;
    // what must start at zero: both bin counts and the error word
    S_CUDA(cudaMemsetAsync(bins[0].count, 0, sizeof(int) * 2 * S_MAX_TILES, st));
    S_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));

    auto part_args = [&](int pin, int pout, int integrate, const Bins &bin_in, const Bins &bin_out) {
        PartArgs a{};
        a.L = L;
        a.ph = ph;
        a.P = P;
        a.bp = bp;
        a.bin_in = bin_in;
        a.bin_out = bin_out;
        a.partial = partial;
        a.pin = pin;
        a.pout = pout;
        a.integrate = integrate;
        a.force = force;
        a.fcol = fcol;
        a.err = err;
        return a;
    };
    if (np > 0) {
        particles_in_kernel<<<(np + 127) / 128, 128, 0, st>>>(particles, P, np, L.nx, L.ny, L.per_x, L.per_y,
                                                              ph.cut_d, err);
        S_CUDA(cudaGetLastError());
        // nothing else runs on a bad particle: f_out and the caller's
        // particles stay as they were
        int h = 0;
        S_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        S_CUDA(cudaStreamSynchronize(st));
        if (h & ERR_BADPARTICLE)
            return sfail(DILBM_ERR_INVALID_ARG, "dilbm_step_static: a particle lies outside the lattice, has a "
                                                "non-finite or non-positive radius or density, non-finite "
                                                "velocities, or a phi tail reaching more than " +
                                                    std::to_string(MAXT) + " tiles; nothing was changed");
        // bin the particles where they are (positions copy 0, bins 0)
        particles_kernel<false><<<(np + PART_WARPS - 1) / PART_WARPS, PART_WARPS * 32, 0, st>>>(part_args(0, 0, 0, bins[0], bins[0]),
                                                                       nullptr, BatchIndex{});
        S_CUDA(cudaGetLastError());
    }

    // ---- the sweep, with the caller's populations (GUARD elements in)
    int dev = 0, sms = 1;
    S_CUDA(cudaGetDevice(&dev));
    S_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = sweep_smem_bytes<float>();
    const long long items = (long long)L.ny * L.ntx;
    long long blocks = 2LL * sms;
    const long long need = (items + SWEEP_WARPS - 1) / SWEEP_WARPS;
    if (blocks > need) blocks = need;
    SweepArgs<float> sa{};
    sa.src = f_in + GUARD;
    sa.dst = f_out + GUARD;
    sa.L = L;
    sa.ph = ph;
    sa.B = bins[0];
    sa.partial = partial;
    sa.clear = np > 0 ? bins[1].count : nullptr;
    sa.err = err;
    if (L.per_x && L.per_y) {
        S_CUDA(cudaFuncSetAttribute(sweep_kernel<float, MODE_STEP, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        sweep_kernel<float, MODE_STEP, false><<<(unsigned)blocks, SWEEP_WARPS * 32, smem, st>>>(sa);
    } else {
        S_CUDA(cudaFuncSetAttribute(sweep_kernel<float, MODE_STEP, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        sweep_kernel<float, MODE_STEP, true><<<(unsigned)blocks, SWEEP_WARPS * 32, smem, st>>>(sa);
    }
    S_CUDA(cudaGetLastError());

    if (np > 0) {
        // force reduction, Wan-Turek, Newton-Euler (positions copy 0 -> 1)
        particles_kernel<false><<<(np + PART_WARPS - 1) / PART_WARPS, PART_WARPS * 32, 0, st>>>(part_args(0, 1, 1, bins[0], bins[1]),
                                                                       nullptr, BatchIndex{});
        S_CUDA(cudaGetLastError());
        particles_out_kernel<<<(np + 127) / 128, 128, 0, st>>>(particles, P, np);
        S_CUDA(cudaGetLastError());
    }

    // ---- device errors: read the error word (a copy into host stack memory)
    int h = 0;
    S_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    S_CUDA(cudaStreamSynchronize(st));
    if (h & ERR_UNSTABLE) return sfail(DILBM_ERR_UNSTABLE, "a node reached rho <= 0 or a non-finite velocity");
    if (h & ERR_TIMEOUT) return sfail(DILBM_ERR_TIMEOUT, "a bounded device wait gave up (1 s)");
    if (h & ERR_OVERFLOW) return sfail(DILBM_ERR_OVERFLOW, "too many particles reach one lattice tile");
    return DILBM_OK;
}

