// C ABI of the DI-LBM library (declared in include/dilbm.h): context
// management, argument checks, and the launch sequence of one time step.
#include "dilbm.h"
#include "dilbm_trace.h"
#include "dilbm_launch.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

using namespace dilbm;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? DILBM_ERR_OOM : DILBM_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define DILBM_CUDA(call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

}  // namespace

struct dilbm_ctx {
    Lattice L{};
    Physics ph{};
    BodyParams bp{};
    int storage = DILBM_FP32;
    int method = DILBM_METHOD_DI;
    size_t elem = 4;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    Particles P{};
    Bins bins[2]{};                   // tile bins by step parity
    float4 *partial = nullptr;        // per tile, slot and row: force / torque partials
    double *force = nullptr, *fcol = nullptr;
    double *fsum = nullptr;           // per particle: sum of (Fx, Fy, T) since the last reset
    long long fsum_steps = 0;
    int *err = nullptr;
    int sticky = 0;
    float *fields = nullptr;          // 4 x nx x ny, allocated on first use
    double *pops = nullptr;           // 9 x nx x ny, allocated on first use
    cudaStream_t stream = nullptr;
    int np = 0;
    int ntiles = 0;
    int num_sms = 1;
    bool timing = false;
    std::vector<cudaEvent_t> ev;      // start/stop pairs around sweep launches
    size_t ev_used = 0;
    long long launches = 0;
    SweepShape shape{};               // launch shape of the step sweep (autotuned or default)
    cudaGraphExec_t g_pair[2] = {nullptr, nullptr};   // two steps from parity 0 / 1, replayed by dilbm_step
    int track = -1;                   // moving frame: tracked particle, -1 when off
    double track_x = 0.0;             // its reference x
    long long *frame_off = nullptr;   // device: columns the frame has moved, allocated on first use
    float *cover = nullptr;           // PS: per-particle covered-area tables (grown by upload_particles)
    // A strip of a lattice decomposed over ranks (dilbm_create_strip): L holds
    // rows [y0, y0 + L.ny) with halo rows across its cuts, Lg the whole
    // lattice (the particles' geometry), tile rows [ty_lo, ty_lo + L.nty).
    bool strip = false;
    int y0 = 0, ty_lo = 0;
    Lattice Lg{};
    void *xsend[2] = {nullptr, nullptr};   // this strip's first / last row (9 plane rows), for the neighbours
    void *xrecv[2] = {nullptr, nullptr};   // the rows just south / north of it (the sweep's halos)
    double *fpart = nullptr;               // per particle: this strip's Fx, Fy, T, repulsion x, y
    bool strip_open = false;               // between dilbm_strip_begin and dilbm_strip_end
    void *owned[40] = {};
    int nowned = 0;
    // dilbm_set_particles packs into pinned host memory, so its copies run
    // asynchronously; up_done marks when the last upload's copies have read it
    void *up_stage = nullptr;
    cudaEvent_t up_done = nullptr;
    // dilbm_forces with the state: one device block in the staging layout
    // (force 3 np, fcol 2 np, x, y, r, ux, uy, omega, theta, rho_s as doubles,
    // then fixed and the error word as ints), read back by one copy
    double *readback = nullptr;
};

// Gathers dilbm_forces' outputs into the readback block (layout above).
__global__ void readback_kernel(double *__restrict__ out, const double *__restrict__ force,
                                const double *__restrict__ fcol, const double *__restrict__ x,
                                const double *__restrict__ y, const double *__restrict__ rest,
                                const int *__restrict__ fixed, const int *__restrict__ err, int np) {
    const long long nd = 13LL * np;
    int *oi = reinterpret_cast<int *>(out + nd);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nd + np + 1;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < 3LL * np) out[i] = force[i];
        else if (i < 5LL * np) out[i] = fcol[i - 3LL * np];
        else if (i < 6LL * np) out[i] = x[i - 5LL * np];
        else if (i < 7LL * np) out[i] = y[i - 6LL * np];
        else if (i < nd) out[i] = rest[i - 7LL * np];
        else if (i < nd + np) oi[i - nd] = fixed[i - nd];
        else oi[np] = *err;
    }
}

namespace {

// Record device memory the context frees at destroy (frees q and fails when
// the table is full).
int keep_owned(dilbm_ctx *c, void *q) {
    if (c->nowned >= (int)(sizeof(c->owned) / sizeof(c->owned[0]))) {
        cudaFree(q);
        return fail(DILBM_ERR_OOM, "too many device allocations for one context");
    }
    c->owned[c->nowned++] = q;
    return DILBM_OK;
}

template <typename Tp>
int dev_alloc(dilbm_ctx *c, Tp **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(Tp) > 0 ? count * sizeof(Tp) : 16);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if (int rc = keep_owned(c, q)) return rc;
    *p = static_cast<Tp *>(q);
    return DILBM_OK;
}

int check_side(const dilbm_side &s, const char *name) {
    if (s.kind < DILBM_SIDE_PERIODIC || s.kind > DILBM_SIDE_PRESSURE)
        return fail(DILBM_ERR_INVALID_ARG, std::string("unknown side kind on ") + name);
    if (s.kind == DILBM_SIDE_PRESSURE && !(s.rho > 0.0))
        return fail(DILBM_ERR_INVALID_ARG, std::string("pressure side needs rho > 0 on ") + name);
    return DILBM_OK;
}

int check_particles(const dilbm_grid *g, const dilbm_particle *p, int np) {
    for (int k = 0; k < np; ++k) {
        const dilbm_particle &q = p[k];
        const bool px = g->west.kind == DILBM_SIDE_PERIODIC, py = g->south.kind == DILBM_SIDE_PERIODIC;
        const bool inx = px ? (q.x >= 0.0 && q.x < g->nx) : (q.x >= 0.0 && q.x <= g->nx - 1);
        const bool iny = py ? (q.y >= 0.0 && q.y < g->ny) : (q.y >= 0.0 && q.y <= g->ny - 1);
        if (!inx || !iny || !(q.r > 0.0) || !(q.rho_s > 0.0) || !std::isfinite(q.r) || !std::isfinite(q.rho_s) ||
            !std::isfinite(q.ux) || !std::isfinite(q.uy) || !std::isfinite(q.omega) || !std::isfinite(q.theta))
            return fail(DILBM_ERR_INVALID_ARG, "particle " + std::to_string(k) +
                                                   " outside the lattice, with a non-positive or non-finite "
                                                   "radius/density, or with non-finite velocities");
    }
    return DILBM_OK;
}

// A tile's nodes share the particle image nearest the tile centre unless the
// periodic axis is shorter than the tile plus two reach radii.
void set_wrap_flags(dilbm_ctx *c, const dilbm_particle *p, int np) {
    double rmax = 0.0;
    for (int k = 0; k < np; ++k) rmax = p[k].r > rmax ? p[k].r : rmax;
    const double reach = 2.0 * (rmax + c->ph.cut_d) + 2.0;
    c->L.wrap_x = c->L.per_x && c->L.nx < reach + TILE_W;
    c->L.wrap_y = c->L.per_y && c->L.ny < reach + TILE_H;
}

// Bytes of the device allocations dilbm_create makes (kept beside it: the
// same arrays, in the same order).
unsigned long long footprint_of(int nx, int ny, size_t elem, int np) {
    const unsigned long long pitch = (unsigned long long)(nx + 31) / 32 * 32;
    const unsigned long long plane = pitch * (unsigned long long)ny;
    const unsigned long long ntiles =
        (unsigned long long)((nx + TILE_W - 1) / TILE_W) * (unsigned long long)((ny + TILE_H - 1) / TILE_H);
    const unsigned long long npa = np > 0 ? (unsigned long long)np : 1ull;
    unsigned long long b = 2ull * (9ull * plane + 2ull * GUARD) * elem;           // populations A, B
    b += 10ull * npa * sizeof(double) + 4ull * npa * sizeof(float) + npa * sizeof(int);   // particle state
    b += 6ull * npa * sizeof(double) + 2ull * npa * sizeof(double) + sizeof(int);         // force, fsum, fcol, err
    b += ntiles * MAXC * TILE_H * sizeof(float4);                                         // partials
    b += 2ull * (ntiles * sizeof(int) + ntiles * MAXC * sizeof(int) + ntiles * MAXC * NREC * sizeof(float4) +
                 npa * MAXT * sizeof(int) + npa * sizeof(int));                           // bins, two parities
    return b;
}

int check_reach(double cut_d, const dilbm_particle *p, int np) {
    // tiles one particle's phi tail may reach must fit the per-particle map
    for (int k = 0; k < np; ++k) {
        const double R = p[k].r + cut_d;
        const long long tx = (long long)std::ceil((2.0 * R + 2.0) / TILE_W) + 1;
        const long long ty = (long long)std::ceil((2.0 * R + 2.0) / TILE_H) + 1;
        if (tx * ty > MAXT)
            return fail(DILBM_ERR_INVALID_ARG, "particle " + std::to_string(k) +
                                                   " is too large: its phi tail would reach more than " +
                                                   std::to_string(MAXT) + " lattice tiles");
    }
    return DILBM_OK;
}

PartArgs particle_args(const dilbm_ctx *c, int cur, int integrate, int phase = 0) {
    const int nxt = integrate ? cur ^ 1 : cur;
    PartArgs a{};
    a.L = c->strip ? c->Lg : c->L;
    if (c->strip) {
        a.ty_lo = c->ty_lo;
        a.ty_hi = c->ty_lo + c->L.nty;
        a.phase = phase;
        a.fpart = c->fpart;
    }
    a.ph = c->ph;
    a.P = c->P;
    a.bp = c->bp;
    a.bin_in = c->bins[cur];
    a.bin_out = c->bins[nxt];
    a.partial = c->partial;
    a.pin = cur;
    a.pout = nxt;
    a.integrate = integrate;
    a.force = c->force;
    a.fcol = c->fcol;
    a.fsum = integrate ? c->fsum : nullptr;
    a.err = c->err;
    a.track = c->track;
    a.track_x = c->track_x;
    return a;
}

int launch_particles(dilbm_ctx *c, int integrate, int phase = 0) {
    const int np = c->np;
    particles_kernel<false><<<(np + PART_WARPS - 1) / PART_WARPS, PART_WARPS * 32, 0, c->stream>>>(
        particle_args(c, c->cur, integrate, phase), nullptr, BatchIndex{});
    DILBM_CUDA(cudaGetLastError());
    c->launches += 1;
    if (c->method == DILBM_METHOD_PS && phase != 1) {
        // the covered-area tables of the positions just written
        const int pout = integrate ? c->cur ^ 1 : c->cur;
        cover_kernel<<<np, dim3(COVER_BX, COVER_BY), 0, c->stream>>>(c->cover, c->P.x[pout], c->P.y[pout], c->P.r, np,
                                                                     c->ph);
        DILBM_CUDA(cudaGetLastError());
        c->launches += 1;
    }
    return DILBM_OK;
}

void drop_graphs(dilbm_ctx *c);

// Rows of shared memory the moving frame's in-place column shift may use.
constexpr size_t FRAME_ROW_BYTES = 48 * 1024;

// The moving frame's column shift of the populations the next step reads,
// decided from the tracked particle's position at the start of this step.
int launch_frame_shift(dilbm_ctx *c) {
    const int blocks = c->L.ny < 2 * c->num_sms ? c->L.ny : 2 * c->num_sms;
    const size_t smem = (size_t)c->L.nx * c->elem;
    void *dst = c->buf[c->cur ^ 1];
    const double *xt = c->P.x[c->cur];
    switch (c->storage) {
    case DILBM_FP32:
        frame_shift_kernel<float><<<blocks, 256, smem, c->stream>>>((float *)dst, c->L, xt, c->track, c->track_x,
                                                                    c->frame_off);
        break;
    case DILBM_FP16_DEV:
        frame_shift_kernel<__half><<<blocks, 256, smem, c->stream>>>((__half *)dst, c->L, xt, c->track, c->track_x,
                                                                     c->frame_off);
        break;
    default:
        frame_shift_kernel<__nv_bfloat16><<<blocks, 256, smem, c->stream>>>((__nv_bfloat16 *)dst, c->L, xt, c->track,
                                                                            c->track_x, c->frame_off);
        break;
    }
    DILBM_CUDA(cudaGetLastError());
    c->launches += 1;
    return DILBM_OK;
}

// PS-LBM: each particle's table of covered cell areas spans the cells within
// K = ceil(r_max + reach) + 1 of its centre cell; grown when a larger radius
// arrives (the particles kernel fills it, the sweep reads it).
int size_cover_tables(dilbm_ctx *c, const dilbm_particle *p, int np) {
    if (c->method != DILBM_METHOD_PS || np == 0) return DILBM_OK;
    double rmax = 0.0;
    for (int k = 0; k < np; ++k) rmax = p[k].r > rmax ? p[k].r : rmax;
    const int K = (int)std::ceil(rmax + c->ph.cut_d) + 1;
    if (K <= c->ph.ck) return DILBM_OK;
    const size_t S = 2 * (size_t)K + 1;
    if (c->cover) {
        DILBM_CUDA(cudaStreamSynchronize(c->stream));
        DILBM_CUDA(cudaFree(c->cover));
        c->cover = nullptr;
    }
    DILBM_CUDA(cudaMalloc(&c->cover, sizeof(float) * S * S * (size_t)np));
    c->ph.ck = K;
    c->bins[0].cover = c->bins[1].cover = c->cover;
    drop_graphs(c);
    return DILBM_OK;
}

int upload_particles(dilbm_ctx *c, const dilbm_particle *p, int np) {
    // every check before any state changes
    int rc = check_reach(c->ph.cut_d, p, np);
    if (rc) return rc;
    const int wx = c->L.wrap_x, wy = c->L.wrap_y;
    set_wrap_flags(c, p, np);
    if (c->L.wrap_x != wx || c->L.wrap_y != wy) drop_graphs(c);
    if ((rc = size_cover_tables(c, p, np))) return rc;
    // pinned staging: x, y, then r, ux, uy, omega, theta, rho_s (one device
    // slice), as doubles, then fixed as ints; reused once the previous
    // upload's copies have read it
    if (!c->up_stage) {
        if (cudaHostAlloc(&c->up_stage, (sizeof(double) * 8 + sizeof(int)) * (size_t)np, cudaHostAllocDefault) != cudaSuccess) {
            c->up_stage = nullptr;
            return fail(DILBM_ERR_OOM, "pinned staging for the particle upload");
        }
        DILBM_CUDA(cudaEventCreateWithFlags(&c->up_done, cudaEventDisableTiming));
    } else {
        DILBM_CUDA(cudaEventSynchronize(c->up_done));
    }
    double *h = static_cast<double *>(c->up_stage);
    int *fx = reinterpret_cast<int *>(h + 8 * (size_t)np);
    for (int k = 0; k < np; ++k) {
        h[0 * np + k] = p[k].x; h[1 * np + k] = p[k].y; h[2 * np + k] = p[k].r;
        h[3 * np + k] = p[k].ux; h[4 * np + k] = p[k].uy; h[5 * np + k] = p[k].omega;
        h[6 * np + k] = p[k].theta; h[7 * np + k] = p[k].rho_s;
        fx[k] = p[k].fixed ? 1 : 0;
    }
    const int cur = c->cur;
    DILBM_CUDA(cudaMemcpyAsync(c->P.x[cur], h, sizeof(double) * np, cudaMemcpyHostToDevice, c->stream));
    DILBM_CUDA(cudaMemcpyAsync(c->P.y[cur], h + np, sizeof(double) * np, cudaMemcpyHostToDevice, c->stream));
    // r, ux, uy, omega, theta, rho_s are consecutive slices of one allocation
    DILBM_CUDA(cudaMemcpyAsync(c->P.r, h + 2 * np, sizeof(double) * 6 * np, cudaMemcpyHostToDevice, c->stream));
    DILBM_CUDA(cudaMemcpyAsync(c->P.fixed, fx, sizeof(int) * np, cudaMemcpyHostToDevice, c->stream));
    DILBM_CUDA(cudaEventRecord(c->up_done, c->stream));
    DILBM_CUDA(cudaMemsetAsync(c->bins[cur].count, 0, sizeof(int) * c->ntiles, c->stream));
    return launch_particles(c, 0);
}

template <typename T>
SweepArgs<T> sweep_args(const dilbm_ctx *c, int cur, const void *src, void *dst, bool clear, FieldsOut fo) {
    SweepArgs<T> a{};
    a.src = (const T *)src;
    a.dst = (T *)dst;
    a.L = c->L;
    a.ph = c->ph;
    a.B = c->np > 0 ? c->bins[cur] : Bins{};     // no particles: no bins to read
    a.partial = c->partial;
    a.clear = (clear && c->np > 0) ? c->bins[cur ^ 1].count : nullptr;
    a.err = c->err;
    a.fo = fo;
    return a;
}

// The FIELDS-mode sweep (dilbm_fields) in the default shape.
template <typename T, bool EDGES, bool PS>
cudaError_t launch_fields_sweep_m(dilbm_ctx *c, const void *src, FieldsOut fo) {
    static int cache[64] = {};
    constexpr size_t smem = sweep_smem_bytes<T>();
    int per_sm = 1;
    cudaError_t e = occupancy_of(sweep_kernel<T, MODE_FIELDS, EDGES, SWEEP_WARPS, PS>, SWEEP_WARPS, smem, cache, &per_sm);
    if (e != cudaSuccess) return e;
    const long long blocks = persistent_grid((long long)c->L.ny * c->L.ntx, SWEEP_WARPS, per_sm, c->num_sms, SweepShape{});
    sweep_kernel<T, MODE_FIELDS, EDGES, SWEEP_WARPS, PS><<<(unsigned)blocks, SWEEP_WARPS * 32, smem, c->stream>>>(
        sweep_args<T>(c, c->cur, src, nullptr, false, fo));
    return cudaGetLastError();
}

template <typename T, bool EDGES>
cudaError_t launch_fields_sweep(dilbm_ctx *c, const void *src, FieldsOut fo) {
    return c->method == DILBM_METHOD_PS ? launch_fields_sweep_m<T, EDGES, true>(c, src, fo)
                                        : launch_fields_sweep_m<T, EDGES, false>(c, src, fo);
}

bool has_edges(const dilbm_ctx *c) { return !(c->L.per_x && c->L.per_y); }

// The step sweep of the current parity in shape `sh` (query: occupancy only).
cudaError_t step_sweep(dilbm_ctx *c, const SweepShape &sh, bool query = false, int *per_sm = nullptr) {
    const void *src = c->buf[c->cur];
    void *dst = c->buf[c->cur ^ 1];
    const bool edges = has_edges(c);
    if (c->method == DILBM_METHOD_PS) {       // the comparison method: default shape only
        if (query) {
            if (per_sm) *per_sm = 1;
            return cudaSuccess;
        }
        switch (c->storage) {
        case DILBM_FP32:
            return launch_step_sweep_ps<float>(sweep_args<float>(c, c->cur, src, dst, true, FieldsOut{}), edges,
                                               c->num_sms, c->stream);
        case DILBM_FP16_DEV:
            return launch_step_sweep_ps<__half>(sweep_args<__half>(c, c->cur, src, dst, true, FieldsOut{}), edges,
                                                c->num_sms, c->stream);
        default:
            return launch_step_sweep_ps<__nv_bfloat16>(
                sweep_args<__nv_bfloat16>(c, c->cur, src, dst, true, FieldsOut{}), edges, c->num_sms, c->stream);
        }
    }
    switch (c->storage) {
    case DILBM_FP32:
        return launch_step_sweep<float>(sweep_args<float>(c, c->cur, src, dst, true, FieldsOut{}), edges, sh,
                                        c->num_sms, c->stream, query, per_sm);
    case DILBM_FP16_DEV:
        return launch_step_sweep<__half>(sweep_args<__half>(c, c->cur, src, dst, true, FieldsOut{}), edges, sh,
                                         c->num_sms, c->stream, query, per_sm);
    default:
        return launch_step_sweep<__nv_bfloat16>(sweep_args<__nv_bfloat16>(c, c->cur, src, dst, true, FieldsOut{}),
                                                edges, sh, c->num_sms, c->stream, query, per_sm);
    }
}

template <int MODE>
int launch_sweep(dilbm_ctx *c, const void *src, void *dst, FieldsOut fo) {
    cudaError_t e;
    if (MODE == MODE_STEP) {
        (void)src;
        (void)dst;
        e = step_sweep(c, c->shape);
    } else {
        const bool edges = has_edges(c);
        switch (c->storage) {
        case DILBM_FP32: e = edges ? launch_fields_sweep<float, true>(c, src, fo) : launch_fields_sweep<float, false>(c, src, fo); break;
        case DILBM_FP16_DEV: e = edges ? launch_fields_sweep<__half, true>(c, src, fo) : launch_fields_sweep<__half, false>(c, src, fo); break;
        default: e = edges ? launch_fields_sweep<__nv_bfloat16, true>(c, src, fo) : launch_fields_sweep<__nv_bfloat16, false>(c, src, fo); break;
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "sweep_kernel launch");
    c->launches += 1;
    return DILBM_OK;
}

int one_step(dilbm_ctx *c) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->timing) {
        if (c->ev_used + 2 > c->ev.size()) {
            for (int k = 0; k < 64; ++k) {
                cudaEvent_t e;
                DILBM_CUDA(cudaEventCreate(&e));
                c->ev.push_back(e);
            }
        }
        e0 = c->ev[c->ev_used];
        e1 = c->ev[c->ev_used + 1];
        c->ev_used += 2;
        DILBM_CUDA(cudaEventRecord(e0, c->stream));
    }
    int rc = launch_sweep<MODE_STEP>(c, c->buf[c->cur], c->buf[c->cur ^ 1], FieldsOut{});
    if (rc) return rc;
    if (c->timing) DILBM_CUDA(cudaEventRecord(e1, c->stream));
    if (c->np > 0 && (rc = launch_particles(c, 1))) return rc;
    if (c->track >= 0 && (rc = launch_frame_shift(c))) return rc;
    c->cur ^= 1;
    c->fsum_steps += 1;
    return DILBM_OK;
}

void drop_graphs(dilbm_ctx *c) {
    for (int p = 0; p < 2; ++p)
        if (c->g_pair[p]) {
            cudaGraphExecDestroy(c->g_pair[p]);
            c->g_pair[p] = nullptr;
        }
}

// Two steps starting at parity p, captured into a graph on the context's
// stream (nothing runs while capturing).
int capture_pair(dilbm_ctx *c, int p) {
    if (c->g_pair[p]) return DILBM_OK;
    const int cur = c->cur;
    const long long l0 = c->launches, f0 = c->fsum_steps;
    c->cur = p;
    cudaGraph_t g = nullptr;
    DILBM_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = one_step(c);
    if (rc == DILBM_OK) rc = one_step(c);
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->cur = cur;
    c->launches = l0;
    c->fsum_steps = f0;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    const cudaError_t e2 = cudaGraphInstantiate(&c->g_pair[p], g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        c->g_pair[p] = nullptr;
        return cuda_fail(e2, "cudaGraphInstantiate");
    }
    return DILBM_OK;
}

// The C ABI code of a lattice's sticky error bits (the first in the order
// UNSTABLE, TIMEOUT, OVERFLOW), and that code with its message.
int sticky_code(int bits) {
    if (bits & ERR_UNSTABLE) return DILBM_ERR_UNSTABLE;
    if (bits & ERR_TIMEOUT) return DILBM_ERR_TIMEOUT;
    if (bits & ERR_OVERFLOW) return DILBM_ERR_OVERFLOW;
    return DILBM_OK;
}

int sticky_error(int bits) {
    switch (sticky_code(bits)) {
    case DILBM_ERR_UNSTABLE: return fail(DILBM_ERR_UNSTABLE, "a node reached rho <= 0 or a non-finite velocity");
    case DILBM_ERR_TIMEOUT: return fail(DILBM_ERR_TIMEOUT, "a bounded device wait gave up (1 s)");
    case DILBM_ERR_OVERFLOW:
        return fail(DILBM_ERR_OVERFLOW, "more than DILBM_MAX_CANDIDATES particles reach one lattice tile");
    default: return DILBM_OK;
    }
}

// Pinned host staging for dilbm_forces: one buffer per host thread, grown on
// demand, so that its copies run asynchronously and the call waits once.
struct PinnedStage {
    void *p = nullptr;
    size_t bytes = 0;
    ~PinnedStage() {
        if (p) cudaFreeHost(p);
    }
    void *get(size_t n) {
        if (n > bytes) {
            if (p) cudaFreeHost(p);
            p = nullptr;
            bytes = 0;
            if (cudaHostAlloc(&p, n, cudaHostAllocDefault) != cudaSuccess) {
                p = nullptr;
                return nullptr;
            }
            bytes = n;
        }
        return p;
    }
};
thread_local PinnedStage t_stage;

int read_sticky(dilbm_ctx *c) {
    int h = 0;
    DILBM_CUDA(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DILBM_CUDA(cudaStreamSynchronize(c->stream));
    c->sticky |= h;
    return sticky_error(c->sticky);
}

}  // namespace

namespace dilbm {
// Lets other translation units of the library report through dilbm_last_error().
int set_last_error(int code, const std::string &msg) { return fail(code, msg); }

// Distance beyond a particle's surface at which its coupling vanishes: the
// phi tail (DI) or the half-diagonal of a cell (PS: a cell whose centre is
// farther than r + sqrt(2)/2 has no covered part).
double reach_cut(int method, double interface_width) {
    return method == DILBM_METHOD_PS ? 0.70711 : PHI_CUT_WIDTHS * interface_width;
}

// Every argument check of dilbm_create (host only; g must not be NULL).
int check_problem(const dilbm_grid *g, dilbm_lattice lattice, double tau, double interface_width,
                  const dilbm_particle *particles, int np) {
    if (lattice != DILBM_D2Q9) return fail(DILBM_ERR_INVALID_ARG, "only DILBM_D2Q9 is supported");
    if (g->nx < 3 || g->ny < 3) return fail(DILBM_ERR_INVALID_ARG, "nx and ny must be >= 3");
    if ((long long)g->nx * g->ny > (1LL << 31)) return fail(DILBM_ERR_INVALID_ARG, "lattice larger than 2^31 nodes");
    if (!(tau > 0.5)) return fail(DILBM_ERR_INVALID_ARG, "tau must be > 0.5");
    if (!(interface_width > 0.0)) return fail(DILBM_ERR_INVALID_ARG, "interface width must be > 0");
    if (np < 0 || (np > 0 && !particles)) return fail(DILBM_ERR_INVALID_ARG, "bad particle array");
    if (g->storage < DILBM_FP32 || g->storage > DILBM_BF16_DEV) return fail(DILBM_ERR_INVALID_ARG, "unknown storage");
    if (g->force_model != DILBM_FORCE_EQ18 && g->force_model != DILBM_FORCE_MOMENTUM)
        return fail(DILBM_ERR_INVALID_ARG, "unknown force model");
    int rc;
    if ((rc = check_side(g->west, "west")) || (rc = check_side(g->east, "east")) ||
        (rc = check_side(g->south, "south")) || (rc = check_side(g->north, "north")))
        return rc;
    if ((g->west.kind == DILBM_SIDE_PERIODIC) != (g->east.kind == DILBM_SIDE_PERIODIC) ||
        (g->south.kind == DILBM_SIDE_PERIODIC) != (g->north.kind == DILBM_SIDE_PERIODIC))
        return fail(DILBM_ERR_INVALID_ARG, "an axis must be periodic on both sides or on neither");
    if (!(g->rho_init > 0.0) || !(g->rho_f > 0.0)) return fail(DILBM_ERR_INVALID_ARG, "densities must be > 0");
    for (int k = 0; k < 5; ++k)
        if (!(g->wan_turek[k] > 0.0)) return fail(DILBM_ERR_INVALID_ARG, "Wan-Turek parameters must be > 0");
    if ((rc = check_particles(g, particles, np))) return rc;
    if (g->method != DILBM_METHOD_DI && g->method != DILBM_METHOD_PS)
        return fail(DILBM_ERR_INVALID_ARG, "unknown coupling method");
    if (g->method == DILBM_METHOD_PS) {
        for (int k = 0; k < np; ++k)
            if (!(particles[k].r >= 1.0))
                return fail(DILBM_ERR_INVALID_ARG, "PS-LBM particles need a radius >= 1 lattice unit");
    }
    return check_reach(reach_cut(g->method, interface_width), particles, np);
}
}  // namespace dilbm

// Failure detection without a fault: one warp waits, with the sweep's bounded
// mbarrier wait, on a shared-memory barrier that no copy and no thread ever
// arrives at.  The wait gives up after its limit and the kernel records
// ERR_TIMEOUT in the caller's error word, as the sweep does, then returns.
__global__ void wait_probe_kernel(int *err, unsigned long long *waited_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncwarp();
    const unsigned long long t0 = global_ns();
    const bool arrived = __all_sync(0xffffffffu, mbar_wait_bounded(&bar, 0));
    if (threadIdx.x == 0) {
        *waited_ns = global_ns() - t0;
        if (!arrived) atomicOr(err, ERR_TIMEOUT);
    }
}

extern "C" {

const char *dilbm_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// A context for rows [y0, y1) of the lattice (the whole lattice: 0, ny).
static int create_ctx(const dilbm_grid *g, dilbm_lattice lattice, double tau, double interface_width,
                      const dilbm_particle *particles, int np, void *cuda_stream, int y0, int y1, dilbm_ctx **out) {
    int rc = dilbm::check_problem(g, lattice, tau, interface_width, particles, np);
    if (rc) return rc;

    dilbm_ctx *c = new dilbm_ctx();
    c->stream = (cudaStream_t)cuda_stream;
    c->np = np;
    c->storage = g->storage;
    c->method = g->method;
    c->elem = g->storage == DILBM_FP32 ? 4 : 2;
    Lattice &L = c->L;
    L.nx = g->nx;
    L.ny = g->ny;
    L.pitch = (g->nx + 31) / 32 * 32;
    L.plane = (long long)L.pitch * L.ny;
    L.ntx = (L.nx + TILE_W - 1) / TILE_W;
    L.nty = (L.ny + TILE_H - 1) / TILE_H;
    L.per_x = g->west.kind == DILBM_SIDE_PERIODIC;
    L.per_y = g->south.kind == DILBM_SIDE_PERIODIC;
    const dilbm_side *sides[4] = {&g->west, &g->east, &g->south, &g->north};
    for (int k = 0; k < 4; ++k) {
        L.side_kind[k] = sides[k]->kind;
        L.side_ux[k] = (float)sides[k]->ux;
        L.side_uy[k] = (float)sides[k]->uy;
        L.side_drho[k] = (float)(sides[k]->rho - 1.0);
    }
    // 16-bit storage: deviations from the initial equilibrium f^eq(rho_init,
    // u0) (Eq. 2), scaled by 2^14 in FP16 so that small values stay normal
    {
        const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
        const bool wide = g->storage == DILBM_FP32;
        const double q = g->storage == DILBM_FP16_DEV ? 1.0 / 16384.0 : 1.0;
        const double r0 = g->rho_init, ux = g->u0[0], uy = g->u0[1];
        for (int i = 0; i < 9; ++i) {
            const double cu = cxof(i) * ux + cyof(i) * uy;
            const double e = w[i] * r0 * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy)) - w[i];
            L.ref_e[i] = wide ? 0.0f : (float)e;
        }
        L.ref_q = (float)q;
        L.ref_iq = (float)(1.0 / q);
        // the reference's moments in the collision's moment form (Eq. 2):
        // m0 = rho - 1, B = rho u0, M = rho u0 u0^T
        const double m[6] = {r0 - 1.0, r0 * ux, r0 * uy, r0 * ux * ux, r0 * uy * uy, r0 * ux * uy};
        for (int k = 0; k < 6; ++k) L.ref_m[k] = wide ? 0.0f : (float)m[k];
    }
    const bool strip = y0 > 0 || y1 < g->ny;
    if (strip) {
        // the particles keep the whole lattice's geometry; the sweep sees
        // rows [y0, y1) with halo rows beyond each cut
        c->strip = true;
        c->Lg = L;
        c->y0 = y0;
        c->ty_lo = y0 / TILE_H;
        const bool cut_s = y0 > 0 || L.per_y, cut_n = y1 < g->ny || L.per_y;
        L.ny = y1 - y0;
        L.plane = (long long)L.pitch * L.ny;
        L.nty = (L.ny + TILE_H - 1) / TILE_H;
        L.per_y = 0;
        if (cut_s) L.side_kind[SOUTH] = SIDE_HALO;
        if (cut_n) L.side_kind[NORTH] = SIDE_HALO;
    }
    c->ntiles = L.ntx * L.nty;
    Physics &ph = c->ph;
    ph.omega = (float)(1.0 / tau);
    ph.kf = (float)(1.0 - 0.5 / tau);
    ph.kforce = g->force_model == DILBM_FORCE_EQ18 ? ph.kf : 1.0f;
    ph.phi_k2 = (float)(-4.0 / (interface_width * std::log(2.0)));
    ph.cut_d = dilbm::reach_cut(g->method, interface_width);
    ph.cut = (float)ph.cut_d;
    if (c->method == DILBM_METHOD_PS) {
        // Eq. 12: the second moment's coupling term is B rho (u_s u_s - u* u*)
        // and the force of Eq. 10 is the momentum the fluid receives
        ph.kf = 1.0f;
        ph.kforce = 1.0f;
    }
    BodyParams &bp = c->bp;
    bp.np = np;
    bp.gx = g->gravity[0];
    bp.gy = g->gravity[1];
    bp.rho_f = g->rho_f;
    bp.eps_p = g->wan_turek[0];
    bp.eps_p2 = g->wan_turek[1];
    bp.eps_w = g->wan_turek[2];
    bp.eps_w2 = g->wan_turek[3];
    bp.xi = g->wan_turek[4];

    auto bail = [&](int code) { dilbm_destroy(c); return code; };
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaDeviceGetAttribute"));
    }
    // each population buffer carries GUARD readable elements on both sides:
    // the sweep stages whole 16-byte-aligned row segments with their halos
    const size_t pop_elems = 9 * (size_t)L.plane + 2 * (size_t)GUARD;
    for (int b = 0; b < 2; ++b) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, pop_elems * c->elem);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc populations"));
        if (int rc = keep_owned(c, q)) return bail(rc);
        c->buf[b] = static_cast<char *>(q) + GUARD * c->elem;
        e = cudaMemsetAsync(q, 0, pop_elems * c->elem, c->stream);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemsetAsync"));
    }
    const int npa = np > 0 ? np : 1;
    double *pd = nullptr;
    float *pf = nullptr;
    if ((rc = dev_alloc(c, &pd, 10 * (size_t)npa)) || (rc = dev_alloc(c, &pf, 4 * (size_t)npa)) ||
        (rc = dev_alloc(c, &c->P.fixed, (size_t)npa)) || (rc = dev_alloc(c, &c->force, 3 * (size_t)npa)) ||
        (rc = dev_alloc(c, &c->fsum, 3 * (size_t)npa)) || (rc = dev_alloc(c, &c->fcol, 2 * (size_t)npa)) ||
        (rc = dev_alloc(c, &c->err, 1)) ||
        (rc = dev_alloc(c, &c->partial, (size_t)c->ntiles * MAXC * TILE_H)))
        return bail(rc);
    for (int b = 0; b < 2; ++b) {
        Bins &B = c->bins[b];
        if ((rc = dev_alloc(c, &B.count, (size_t)c->ntiles)) || (rc = dev_alloc(c, &B.ids, (size_t)c->ntiles * MAXC)) ||
            (rc = dev_alloc(c, &B.rec, (size_t)c->ntiles * MAXC * NREC)) ||
            (rc = dev_alloc(c, &B.pslot, (size_t)npa * MAXT)) || (rc = dev_alloc(c, &B.npslot, (size_t)npa)))
            return bail(rc);
    }
    c->P.x[0] = pd; c->P.x[1] = pd + npa; c->P.y[0] = pd + 2 * npa; c->P.y[1] = pd + 3 * npa;
    c->P.r = pd + 4 * npa; c->P.ux = pd + 5 * npa; c->P.uy = pd + 6 * npa; c->P.omega = pd + 7 * npa;
    c->P.theta = pd + 8 * npa; c->P.rho_s = pd + 9 * npa;
    c->P.xf[0] = pf; c->P.xf[1] = pf + npa; c->P.yf[0] = pf + 2 * npa; c->P.yf[1] = pf + 3 * npa;
    if (c->strip) {
        // exchange buffers: 9 plane rows each, GUARD readable elements around
        const size_t row_elems = 9 * (size_t)L.pitch + 2 * (size_t)GUARD;
        for (int k = 0; k < 4; ++k) {
            void *q = nullptr;
            cudaError_t e2 = cudaMalloc(&q, row_elems * c->elem);
            if (e2 != cudaSuccess) return bail(cuda_fail(e2, "cudaMalloc halo rows"));
            if (int rc = keep_owned(c, q)) return bail(rc);
            e2 = cudaMemsetAsync(q, 0, row_elems * c->elem, c->stream);
            if (e2 != cudaSuccess) return bail(cuda_fail(e2, "cudaMemsetAsync"));
            (k < 2 ? c->xsend[k] : c->xrecv[k - 2]) = static_cast<char *>(q) + GUARD * c->elem;
        }
        if ((rc = dev_alloc(c, &c->fpart, 5 * (size_t)npa))) return bail(rc);
        if (L.side_kind[SOUTH] == SIDE_HALO) L.halo[0] = c->xrecv[0];
        if (L.side_kind[NORTH] == SIDE_HALO) L.halo[1] = c->xrecv[1];
    }
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->force, 0, sizeof(double) * 3 * npa, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->fsum, 0, sizeof(double) * 3 * npa, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->fcol, 0, sizeof(double) * 2 * npa, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->bins[0].count, 0, sizeof(int) * c->ntiles, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->bins[1].count, 0, sizeof(int) * c->ntiles, c->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMemsetAsync"));
    // uniform initial state f^eq(rho_init, u0)
    const int blocks = 152 * 8;
    const float drho = (float)(g->rho_init - 1.0), u0x = (float)g->u0[0], u0y = (float)g->u0[1];
    switch (c->storage) {
    case DILBM_FP32: init_kernel<float><<<blocks, 256, 0, c->stream>>>((float *)c->buf[0], L, drho, u0x, u0y); break;
    case DILBM_FP16_DEV: init_kernel<__half><<<blocks, 256, 0, c->stream>>>((__half *)c->buf[0], L, drho, u0x, u0y); break;
    default: init_kernel<__nv_bfloat16><<<blocks, 256, 0, c->stream>>>((__nv_bfloat16 *)c->buf[0], L, drho, u0x, u0y); break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(e, "init_kernel"));
    c->launches += 1;
    for (int k = 0; k < 2 && c->strip; ++k) {
        // the neighbours' rows start in the same uniform state
        Lattice Lh = L;
        Lh.ny = 1;
        Lh.plane = L.pitch;
        switch (c->storage) {
        case DILBM_FP32: init_kernel<float><<<64, 256, 0, c->stream>>>((float *)c->xrecv[k], Lh, drho, u0x, u0y); break;
        case DILBM_FP16_DEV: init_kernel<__half><<<64, 256, 0, c->stream>>>((__half *)c->xrecv[k], Lh, drho, u0x, u0y); break;
        default: init_kernel<__nv_bfloat16><<<64, 256, 0, c->stream>>>((__nv_bfloat16 *)c->xrecv[k], Lh, drho, u0x, u0y); break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(e, "init_kernel"));
        c->launches += 1;
    }
    if (np > 0 && (rc = upload_particles(c, particles, np))) return bail(rc);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(cuda_fail(e, "cudaStreamSynchronize"));
    *out = c;
    return DILBM_OK;
}

extern "C" {

int dilbm_create(const dilbm_grid *g, dilbm_lattice lattice, double tau, double interface_width,
                 const dilbm_particle *particles, int np, void *cuda_stream, dilbm_ctx **out) {
    const dilbm::TraceRange trace("dilbm_create");
    if (!g || !out) return fail(DILBM_ERR_INVALID_ARG, "grid and out must not be NULL");
    *out = nullptr;
    return create_ctx(g, lattice, tau, interface_width, particles, np, cuda_stream, 0, g->ny, out);
}

int dilbm_create_strip(const dilbm_grid *g, dilbm_lattice lattice, double tau, double interface_width,
                       const dilbm_particle *particles, int np, int y0, int y1, void *cuda_stream,
                       dilbm_ctx **out) {
    const dilbm::TraceRange trace("dilbm_create_strip");
    if (!g || !out) return fail(DILBM_ERR_INVALID_ARG, "grid and out must not be NULL");
    *out = nullptr;
    if (y0 < 0 || y1 > g->ny || y1 - y0 < 2 || (y0 == 0 && y1 == g->ny))
        return fail(DILBM_ERR_INVALID_ARG, "a strip holds rows [y0, y1) with 0 <= y0, y1 <= ny, at least two rows "
                                           "and not the whole lattice");
    if (y0 % TILE_H != 0 || (y1 % TILE_H != 0 && y1 != g->ny))
        return fail(DILBM_ERR_INVALID_ARG, "strip cuts must lie on multiples of " + std::to_string(TILE_H) + " rows");
    if (g->south.kind == DILBM_SIDE_PERIODIC && np > 0) {
        double rmax = 0.0;
        for (int k = 0; k < np && particles; ++k) rmax = particles[k].r > rmax ? particles[k].r : rmax;
        const double reach = 2.0 * (rmax + dilbm::reach_cut(g->method, interface_width)) + 2.0;
        if (g->ny < reach + TILE_H)
            return fail(DILBM_ERR_INVALID_ARG, "a periodic y axis this short for its discs is not split into strips");
    }
    return create_ctx(g, lattice, tau, interface_width, particles, np, cuda_stream, y0, y1, out);
}

int dilbm_strip_begin(dilbm_ctx *c) {
    const dilbm::TraceRange trace("dilbm_strip_begin");
    if (!c || !c->strip || c->strip_open) return fail(DILBM_ERR_INVALID_ARG, "not a strip, or a step already begun");
    int rc = launch_sweep<MODE_STEP>(c, c->buf[c->cur], c->buf[c->cur ^ 1], FieldsOut{});
    if (rc) return rc;
    if (c->np > 0 && (rc = launch_particles(c, 1, 1))) return rc;
    // this strip's first and last rows of every plane, for the neighbours
    const size_t pitch_b = (size_t)c->L.pitch * c->elem, plane_b = (size_t)c->L.plane * c->elem;
    const char *dst = static_cast<const char *>(c->buf[c->cur ^ 1]);
    DILBM_CUDA(cudaMemcpy2DAsync(c->xsend[0], pitch_b, dst, plane_b, pitch_b, 9, cudaMemcpyDeviceToDevice, c->stream));
    DILBM_CUDA(cudaMemcpy2DAsync(c->xsend[1], pitch_b, dst + (size_t)(c->L.ny - 1) * pitch_b, plane_b, pitch_b, 9,
                                 cudaMemcpyDeviceToDevice, c->stream));
    c->strip_open = true;
    return DILBM_OK;
}

int dilbm_strip_end(dilbm_ctx *c) {
    const dilbm::TraceRange trace("dilbm_strip_end");
    if (!c || !c->strip || !c->strip_open) return fail(DILBM_ERR_INVALID_ARG, "not a strip, or no step begun");
    int rc;
    if (c->np > 0 && (rc = launch_particles(c, 1, 2))) return rc;
    c->cur ^= 1;
    c->fsum_steps += 1;
    c->strip_open = false;
    return DILBM_OK;
}

int dilbm_strip_buffers(dilbm_ctx *c, double **fpart, void **send_south, void **send_north, void **recv_south,
                        void **recv_north, long long *row_elems) {
    if (!c || !c->strip) return fail(DILBM_ERR_INVALID_ARG, "not a strip");
    if (fpart) *fpart = c->fpart;
    if (send_south) *send_south = c->xsend[0];
    if (send_north) *send_north = c->xsend[1];
    if (recv_south) *recv_south = c->xrecv[0];
    if (recv_north) *recv_north = c->xrecv[1];
    if (row_elems) *row_elems = 9LL * c->L.pitch;
    return DILBM_OK;
}

int dilbm_step(dilbm_ctx *c, long long nsteps) {
    const dilbm::TraceRange trace("dilbm_step");
    if (!c || nsteps < 0) return fail(DILBM_ERR_INVALID_ARG, "bad context or step count");
    if (c->strip) return fail(DILBM_ERR_INVALID_ARG, "a strip steps through dilbm_strip_begin / dilbm_strip_end");
    // whole step pairs replay a captured graph (timing brackets every sweep
    // launch with events instead; a stream the caller is capturing gets the
    // launches themselves)
    bool graphs = !c->timing && nsteps >= 2 && c->stream != nullptr && c->stream != cudaStreamLegacy;
    if (graphs) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        graphs = cudaStreamIsCapturing(c->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
    }
    long long t = 0;
    if (graphs) {
        int rc = capture_pair(c, c->cur);
        if (rc) return rc;
        for (; t + 2 <= nsteps; t += 2) DILBM_CUDA(cudaGraphLaunch(c->g_pair[c->cur], c->stream));
        c->launches += t * ((c->np > 0 ? (c->method == DILBM_METHOD_PS ? 3 : 2) : 1) + (c->track >= 0 ? 1 : 0));
        c->fsum_steps += t;
    }
    for (; t < nsteps; ++t) {
        int rc = one_step(c);
        if (rc) return rc;
    }
    return DILBM_OK;
}

int dilbm_sync(dilbm_ctx *c) {
    if (!c) return fail(DILBM_ERR_INVALID_ARG, "NULL context");
    return read_sticky(c);
}

int dilbm_forces(dilbm_ctx *c, double *force, double *fcol, dilbm_particle *state) {
    if (!c) return fail(DILBM_ERR_INVALID_ARG, "NULL context");
    if (c->np > 0 && !force) return fail(DILBM_ERR_INVALID_ARG, "force must not be NULL");
    const size_t np = (size_t)c->np;
    if (np == 0) return read_sticky(c);
    // staged: force (3 np), fcol (2 np), x, y, r, ux, uy, omega, theta, rho_s
    // (8 np) as doubles, then fixed (np) and the error word as ints
    double *h = static_cast<double *>(t_stage.get(sizeof(double) * 13 * np + sizeof(int) * (np + 1)));
    if (!h) return fail(DILBM_ERR_OOM, "pinned staging for dilbm_forces");
    double *hf = h, *hc = h + 3 * np, *hs = h + 5 * np;
    int *fx = reinterpret_cast<int *>(h + 13 * np), *herr = fx + np;
    const size_t block_bytes = sizeof(double) * 13 * np + sizeof(int) * (np + 1);
    if (state) {
        // everything in one copy, gathered on the device
        if (!c->readback) {
            void *q = nullptr;
            if (cudaMalloc(&q, block_bytes) != cudaSuccess) return fail(DILBM_ERR_OOM, "device readback block for dilbm_forces");
            c->readback = static_cast<double *>(q);
        }
        const int threads = 256, blocks = (int)((block_bytes / sizeof(int) + threads - 1) / threads);
        readback_kernel<<<blocks < 4 * c->num_sms ? blocks : 4 * c->num_sms, threads, 0, c->stream>>>(
            c->readback, c->force, c->fcol, c->P.x[c->cur], c->P.y[c->cur], c->P.r, c->P.fixed, c->err, (int)np);
        DILBM_CUDA(cudaGetLastError());
        c->launches += 1;
        DILBM_CUDA(cudaMemcpyAsync(h, c->readback, block_bytes, cudaMemcpyDeviceToHost, c->stream));
    } else {
        DILBM_CUDA(cudaMemcpyAsync(hf, c->force, sizeof(double) * 3 * np, cudaMemcpyDeviceToHost, c->stream));
        if (fcol) DILBM_CUDA(cudaMemcpyAsync(hc, c->fcol, sizeof(double) * 2 * np, cudaMemcpyDeviceToHost, c->stream));
        DILBM_CUDA(cudaMemcpyAsync(herr, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    }
    DILBM_CUDA(cudaStreamSynchronize(c->stream));
    c->sticky |= *herr;
    std::memcpy(force, hf, sizeof(double) * 3 * np);
    if (fcol) std::memcpy(fcol, hc, sizeof(double) * 2 * np);
    if (state) {
        for (size_t k = 0; k < np; ++k) {
            dilbm_particle &q = state[k];
            q.x = hs[k]; q.y = hs[np + k]; q.r = hs[2 * np + k]; q.ux = hs[3 * np + k]; q.uy = hs[4 * np + k];
            q.omega = hs[5 * np + k]; q.theta = hs[6 * np + k]; q.rho_s = hs[7 * np + k]; q.fixed = fx[k];
        }
    }
    return sticky_error(c->sticky);
}

int dilbm_force_mean(dilbm_ctx *c, double *mean, long long *nsteps) {
    if (!c || !nsteps || (c->np > 0 && !mean)) return fail(DILBM_ERR_INVALID_ARG, "NULL argument");
    const int np = c->np;
    *nsteps = c->fsum_steps;
    if (np == 0) return read_sticky(c);
    DILBM_CUDA(cudaMemcpyAsync(mean, c->fsum, sizeof(double) * 3 * np, cudaMemcpyDeviceToHost, c->stream));
    const int rc = read_sticky(c);   // synchronises the stream
    const double inv = c->fsum_steps > 0 ? 1.0 / (double)c->fsum_steps : 0.0;
    for (int k = 0; k < 3 * np; ++k) mean[k] *= inv;
    return rc;
}

int dilbm_set_moving_frame(dilbm_ctx *c, int particle, double x_ref) {
    if (!c) return fail(DILBM_ERR_INVALID_ARG, "NULL context");
    if (c->strip && particle >= 0) return fail(DILBM_ERR_INVALID_ARG, "moving frame: not on a strip");
    if (particle < -1 || particle >= c->np)
        return fail(DILBM_ERR_INVALID_ARG, "moving frame: particle index out of range");
    if (particle >= 0 && !std::isfinite(x_ref)) return fail(DILBM_ERR_INVALID_ARG, "moving frame: x_ref not finite");
    if (particle >= 0 && (size_t)c->L.nx * c->elem > FRAME_ROW_BYTES)
        return fail(DILBM_ERR_INVALID_ARG, "moving frame: a row of nx populations exceeds " +
                                               std::to_string(FRAME_ROW_BYTES) + " bytes");
    if (!c->frame_off) {
        int rc = dev_alloc(c, &c->frame_off, 1);
        if (rc) return rc;
        DILBM_CUDA(cudaMemsetAsync(c->frame_off, 0, sizeof(long long), c->stream));
    }
    c->track = particle;
    c->track_x = particle >= 0 ? x_ref : 0.0;
    drop_graphs(c);
    return DILBM_OK;
}

int dilbm_frame_offset(dilbm_ctx *c, long long *offset) {
    if (!c || !offset) return fail(DILBM_ERR_INVALID_ARG, "NULL argument");
    *offset = 0;
    if (!c->frame_off) return DILBM_OK;
    DILBM_CUDA(cudaMemcpyAsync(offset, c->frame_off, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    DILBM_CUDA(cudaStreamSynchronize(c->stream));
    return DILBM_OK;
}

int dilbm_wait_probe(void *cuda_stream, double *waited_seconds) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    void *q = nullptr;
    DILBM_CUDA(cudaMalloc(&q, 16));
    int *err = static_cast<int *>(q);
    unsigned long long *waited = reinterpret_cast<unsigned long long *>(static_cast<char *>(q) + 8);
    cudaError_t e = cudaMemsetAsync(q, 0, 16, st);
    if (e == cudaSuccess) {
        wait_probe_kernel<<<1, 32, 0, st>>>(err, waited);
        e = cudaGetLastError();
    }
    int h_err = 0;
    unsigned long long h_ns = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_ns, waited, sizeof(h_ns), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(q);
    if (e != cudaSuccess) return cuda_fail(e, "dilbm_wait_probe");
    if (waited_seconds) *waited_seconds = (double)h_ns * 1e-9;
    if (h_err & ERR_TIMEOUT) return fail(DILBM_ERR_TIMEOUT, "bounded device wait gave up (as intended by the probe)");
    return DILBM_OK;
}

int dilbm_force_mean_reset(dilbm_ctx *c) {
    if (!c) return fail(DILBM_ERR_INVALID_ARG, "NULL context");
    if (c->np > 0) DILBM_CUDA(cudaMemsetAsync(c->fsum, 0, sizeof(double) * 3 * c->np, c->stream));
    c->fsum_steps = 0;
    return DILBM_OK;
}

int dilbm_fields(dilbm_ctx *c, float *rho, float *ux, float *uy, float *phi, int on_device) {
    if (!c) return fail(DILBM_ERR_INVALID_ARG, "NULL context");
    const size_t n = (size_t)c->L.nx * c->L.ny;
    FieldsOut fo{};
    if (on_device) {
        fo = FieldsOut{rho, ux, uy, phi};
        return launch_sweep<MODE_FIELDS>(c, c->buf[c->cur], nullptr, fo);
    }
    if (!c->fields) {
        void *q = nullptr;
        DILBM_CUDA(cudaMalloc(&q, sizeof(float) * 4 * n));
        if (int rc = keep_owned(c, q)) return rc;
        c->fields = (float *)q;
    }
    fo = FieldsOut{c->fields, c->fields + n, c->fields + 2 * n, c->fields + 3 * n};
    int rc = launch_sweep<MODE_FIELDS>(c, c->buf[c->cur], nullptr, fo);
    if (rc) return rc;
    float *dst[4] = {rho, ux, uy, phi};
    for (int k = 0; k < 4; ++k)
        if (dst[k]) DILBM_CUDA(cudaMemcpyAsync(dst[k], c->fields + k * n, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
    DILBM_CUDA(cudaStreamSynchronize(c->stream));
    return DILBM_OK;
}

static int ensure_pops(dilbm_ctx *c) {
    if (c->pops) return DILBM_OK;
    void *q = nullptr;
    DILBM_CUDA(cudaMalloc(&q, sizeof(double) * 9 * (size_t)c->L.nx * c->L.ny));
    if (int rc = keep_owned(c, q)) return rc;
    c->pops = (double *)q;
    return DILBM_OK;
}

int dilbm_get_populations(dilbm_ctx *c, double *f) {
    if (!c || !f) return fail(DILBM_ERR_INVALID_ARG, "NULL argument");
    int rc = ensure_pops(c);
    if (rc) return rc;
    const int blocks = 152 * 8;
    switch (c->storage) {
    case DILBM_FP32: export_kernel<float><<<blocks, 256, 0, c->stream>>>((const float *)c->buf[c->cur], c->L, c->pops); break;
    case DILBM_FP16_DEV: export_kernel<__half><<<blocks, 256, 0, c->stream>>>((const __half *)c->buf[c->cur], c->L, c->pops); break;
    default: export_kernel<__nv_bfloat16><<<blocks, 256, 0, c->stream>>>((const __nv_bfloat16 *)c->buf[c->cur], c->L, c->pops); break;
    }
    DILBM_CUDA(cudaGetLastError());
    c->launches += 1;
    DILBM_CUDA(cudaMemcpyAsync(f, c->pops, sizeof(double) * 9 * (size_t)c->L.nx * c->L.ny, cudaMemcpyDeviceToHost, c->stream));
    DILBM_CUDA(cudaStreamSynchronize(c->stream));
    return DILBM_OK;
}

int dilbm_set_populations(dilbm_ctx *c, const double *f) {
    if (!c || !f) return fail(DILBM_ERR_INVALID_ARG, "NULL argument");
    int rc = ensure_pops(c);
    if (rc) return rc;
    DILBM_CUDA(cudaMemcpyAsync(c->pops, f, sizeof(double) * 9 * (size_t)c->L.nx * c->L.ny, cudaMemcpyHostToDevice, c->stream));
    const int blocks = 152 * 8;
    switch (c->storage) {
    case DILBM_FP32: import_kernel<float><<<blocks, 256, 0, c->stream>>>((float *)c->buf[c->cur], c->L, c->pops); break;
    case DILBM_FP16_DEV: import_kernel<__half><<<blocks, 256, 0, c->stream>>>((__half *)c->buf[c->cur], c->L, c->pops); break;
    default: import_kernel<__nv_bfloat16><<<blocks, 256, 0, c->stream>>>((__nv_bfloat16 *)c->buf[c->cur], c->L, c->pops); break;
    }
    DILBM_CUDA(cudaGetLastError());
    c->launches += 1;
    DILBM_CUDA(cudaStreamSynchronize(c->stream));
    return DILBM_OK;
}

int dilbm_set_particles(dilbm_ctx *c, const dilbm_particle *p, int np) {
    if (!c || np != c->np || (np > 0 && !p)) return fail(DILBM_ERR_INVALID_ARG, "particle count differs from create");
    dilbm_grid g{};
    g.nx = c->L.nx;
    g.ny = c->L.ny;
    g.west.kind = g.east.kind = c->L.per_x ? DILBM_SIDE_PERIODIC : DILBM_SIDE_VELOCITY;
    g.south.kind = g.north.kind = c->L.per_y ? DILBM_SIDE_PERIODIC : DILBM_SIDE_VELOCITY;
    int rc = check_particles(&g, p, np);
    if (rc) return rc;
    return np > 0 ? upload_particles(c, p, np) : DILBM_OK;
}

void dilbm_destroy(dilbm_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (int k = 0; k < c->nowned; ++k) cudaFree(c->owned[k]);
    if (c->cover) cudaFree(c->cover);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->up_done) cudaEventDestroy(c->up_done);
    if (c->up_stage) cudaFreeHost(c->up_stage);
    if (c->readback) cudaFree(c->readback);
    delete c;
}

int dilbm_set_timing(dilbm_ctx *c, int enable) {
    if (!c) return fail(DILBM_ERR_INVALID_ARG, "NULL context");
    DILBM_CUDA(cudaStreamSynchronize(c->stream));
    c->timing = enable != 0;
    c->ev_used = 0;
    return DILBM_OK;
}

int dilbm_sweep_time(dilbm_ctx *c, double *ms_total, long long *launches) {
    if (!c || !ms_total || !launches) return fail(DILBM_ERR_INVALID_ARG, "NULL argument");
    DILBM_CUDA(cudaStreamSynchronize(c->stream));
    double total = 0.0;
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
        float ms = 0.f;
        DILBM_CUDA(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
        total += ms;
    }
    *ms_total = total;
    *launches = (long long)(c->ev_used / 2);
    return DILBM_OK;
}

long long dilbm_launch_count(const dilbm_ctx *c) { return c ? c->launches : -1; }

int dilbm_footprint(const dilbm_grid *g, int np, unsigned long long *bytes) {
    if (!g || !bytes || np < 0 || g->nx < 3 || g->ny < 3 || g->storage < DILBM_FP32 || g->storage > DILBM_BF16_DEV)
        return fail(DILBM_ERR_INVALID_ARG, "dilbm_footprint: bad grid, particle count or output pointer");
    *bytes = footprint_of(g->nx, g->ny, g->storage == DILBM_FP32 ? 4 : 2, np);
    return DILBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batches
// Many lattices advanced together: one sweep launch over the concatenated row
// segments of every member and one particle launch over all their particles
// per step, replayed from CUDA graphs.
struct dilbm_batch {
    std::vector<dilbm_ctx *> members;
    std::vector<int> cur0;              // members' parity when the launches were captured
    int storage = DILBM_FP32;
    long long done = 0;                 // batch steps since the capture
    cudaStream_t stream = nullptr;      // private stream the graphs run on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<cudaStream_t> member_streams;
    std::vector<void *> sweep_params[2];   // BatchArgs<T> per launch group, per phase (host copies)
    PartArgs *part_args[2] = {nullptr, nullptr};
    int *part_start = nullptr;          // n + 1
    int *const *err_ptrs = nullptr;     // device: every member's error word
    int *err_out = nullptr;             // device: their values, gathered for one copy
    std::vector<int> err_host;
    int nparts = 0;
    SweepShape shape{};                 // launch shape of the batched sweep
    cudaGraphExec_t g_pair = nullptr, g_single[2] = {nullptr, nullptr};
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    long long launches = 0;
};

namespace {

constexpr int MAX_BATCH = 1024;

// Copies every member's error word into one array, so that a batch sync
// reads them all with a single device-to-host copy.
__global__ void gather_errors_kernel(int *const *__restrict__ err, int n, int *__restrict__ out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) out[k] = *err[k];
}

void free_sweep_params(dilbm_batch *b) {
    for (int phase = 0; phase < 2; ++phase) {
        for (void *q : b->sweep_params[phase]) std::free(q);
        b->sweep_params[phase].clear();
    }
}

// Host copies of the batched sweep's parameters: members in groups of at
// most BATCH_LAUNCH_MAX, both phases (the second step of a pair runs every
// member at the other parity).
template <typename T>
void build_sweep_params(dilbm_batch *b) {
    free_sweep_params(b);
    const int n = (int)b->members.size();
    for (int g0 = 0; g0 < n; g0 += BATCH_LAUNCH_MAX) {
        const int gn = n - g0 < BATCH_LAUNCH_MAX ? n - g0 : BATCH_LAUNCH_MAX;
        for (int phase = 0; phase < 2; ++phase) {
            BatchArgs<T> *ba = static_cast<BatchArgs<T> *>(std::calloc(1, sizeof(BatchArgs<T>)));
            ba->n = gn;
            ba->item_start[0] = ba->tile_start[0] = 0;
            for (int k = 0; k < gn; ++k) {
                const dilbm_ctx *c = b->members[g0 + k];
                const int cur = b->cur0[g0 + k] ^ phase;
                ba->a[k] = sweep_args<T>(c, cur, c->buf[cur], c->buf[cur ^ 1], true, FieldsOut{});
                ba->item_start[k + 1] = ba->item_start[k] + c->L.ny * c->L.ntx;
                ba->tile_start[k + 1] = ba->tile_start[k] + c->L.ntx * c->L.nty;
            }
            b->sweep_params[phase].push_back(ba);
        }
    }
}

int upload_part_args(dilbm_batch *b) {
    const size_t n = b->members.size();
    for (int phase = 0; phase < 2; ++phase) {
        std::vector<PartArgs> pa(n);
        for (size_t k = 0; k < n; ++k) pa[k] = particle_args(b->members[k], b->cur0[k] ^ phase, 1);
        DILBM_CUDA(cudaMemcpyAsync(b->part_args[phase], pa.data(), sizeof(PartArgs) * n, cudaMemcpyHostToDevice, b->stream));
        DILBM_CUDA(cudaStreamSynchronize(b->stream));
    }
    return DILBM_OK;
}

template <typename T>
cudaError_t batch_sweep_groups(dilbm_batch *b, int phase, const SweepShape &sh) {
    const int num_sms = b->members[0]->num_sms;
    for (size_t g = 0; g < b->sweep_params[phase].size(); ++g) {
        const BatchArgs<T> &ba = *static_cast<const BatchArgs<T> *>(b->sweep_params[phase][g]);
        cudaError_t e = launch_batch_sweep<T>(ba, sh, num_sms, b->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Every launch group of the batched sweep at `phase` in shape `sh`.
cudaError_t batch_sweep(dilbm_batch *b, int phase, const SweepShape &sh) {
    if (b->storage == DILBM_FP32) return batch_sweep_groups<float>(b, phase, sh);
    if (b->storage == DILBM_FP16_DEV) return batch_sweep_groups<__half>(b, phase, sh);
    return batch_sweep_groups<__nv_bfloat16>(b, phase, sh);
}

// One batch step at `phase`: the sweep over every member, then the particles.
int batch_phase(dilbm_batch *b, int phase) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (b->timing) {
        if (b->ev_used + 2 > b->ev.size())
            for (int k = 0; k < 64; ++k) {
                cudaEvent_t e;
                DILBM_CUDA(cudaEventCreate(&e));
                b->ev.push_back(e);
            }
        e0 = b->ev[b->ev_used];
        e1 = b->ev[b->ev_used + 1];
        b->ev_used += 2;
        DILBM_CUDA(cudaEventRecord(e0, b->stream));
    }
    cudaError_t e = batch_sweep(b, phase, b->shape);
    if (e != cudaSuccess) return cuda_fail(e, "batched sweep_kernel launch");
    if (b->timing) DILBM_CUDA(cudaEventRecord(e1, b->stream));
    b->launches += (long long)b->sweep_params[phase].size();
    if (b->nparts > 0) {
        BatchIndex pi{b->part_start, nullptr, (int)b->members.size()};
        particles_kernel<true><<<(b->nparts + PART_WARPS - 1) / PART_WARPS, PART_WARPS * 32, 0, b->stream>>>(PartArgs{}, b->part_args[phase], pi);
        DILBM_CUDA(cudaGetLastError());
        b->launches += 1;
    }
    return DILBM_OK;
}

int capture(dilbm_batch *b, int first_phase, int nphases, cudaGraphExec_t *out) {
    if (*out) {
        cudaGraphExecDestroy(*out);
        *out = nullptr;
    }
    cudaGraph_t g = nullptr;
    const long long l0 = b->launches;
    DILBM_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = DILBM_OK;
    for (int k = 0; k < nphases && rc == DILBM_OK; ++k) rc = batch_phase(b, (first_phase + k) & 1);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    b->launches = l0;    // capturing launches nothing
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return DILBM_OK;
}

// (Re)build every launch of the batch from the members' current parity:
// sweep parameters, particle descriptors and the three graphs.
int prepare_batch(dilbm_batch *b) {
    for (size_t k = 0; k < b->members.size(); ++k) b->cur0[k] = b->members[k]->cur;
    b->done = 0;
    if (b->storage == DILBM_FP32) build_sweep_params<float>(b);
    else if (b->storage == DILBM_FP16_DEV) build_sweep_params<__half>(b);
    else build_sweep_params<__nv_bfloat16>(b);
    int rc;
    if ((rc = upload_part_args(b))) return rc;
    if ((rc = capture(b, 0, 2, &b->g_pair)) || (rc = capture(b, 0, 1, &b->g_single[0])) ||
        (rc = capture(b, 1, 1, &b->g_single[1])))
        return rc;
    return DILBM_OK;
}

// Kernels launched by one batch step (sweep groups + particles).
int batch_launches_per_step(const dilbm_batch *b) {
    return (int)b->sweep_params[0].size() + (b->nparts > 0 ? 1 : 0);
}

}  // namespace

extern "C" {

int dilbm_batch_create(dilbm_ctx *const *members, int n, void *cuda_stream, dilbm_batch **out) {
    (void)cuda_stream;
    if (!members || !out || n < 1 || n > MAX_BATCH)
        return fail(DILBM_ERR_INVALID_ARG, "a batch takes 1.." + std::to_string(MAX_BATCH) + " contexts");
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (!members[k]) return fail(DILBM_ERR_INVALID_ARG, "NULL member context");
        if (members[k]->storage != members[0]->storage)
            return fail(DILBM_ERR_INVALID_ARG, "all members of a batch must use the same storage");
        if (members[k]->method != DILBM_METHOD_DI)
            return fail(DILBM_ERR_INVALID_ARG, "batches advance DI-LBM contexts only");
        if (members[k]->strip)
            return fail(DILBM_ERR_INVALID_ARG, "a strip of a decomposed lattice cannot join a batch");
        if (members[k]->track >= 0)
            return fail(DILBM_ERR_INVALID_ARG, "batches advance fixed-frame contexts only");
        for (int j = 0; j < k; ++j)
            if (members[j] == members[k]) return fail(DILBM_ERR_INVALID_ARG, "a context appears twice in the batch");
    }
    dilbm_batch *b = new dilbm_batch();
    auto bail = [&](int code) { dilbm_batch_destroy(b); return code; };
    b->members.assign(members, members + n);
    b->cur0.resize(n);
    b->storage = members[0]->storage;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess)
        return bail(cuda_fail(e, "batch stream/events"));
    for (int k = 0; k < n; ++k) {
        bool seen = false;
        for (cudaStream_t s : b->member_streams) seen |= s == members[k]->stream;
        if (!seen) b->member_streams.push_back(members[k]->stream);
    }
    // particles of each member, in one list
    std::vector<int> ps(n + 1, 0);
    for (int k = 0; k < n; ++k) ps[k + 1] = ps[k] + members[k]->np;
    b->nparts = ps[n];
    for (int phase = 0; phase < 2; ++phase)
        if ((e = cudaMalloc((void **)&b->part_args[phase], sizeof(PartArgs) * n)) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMalloc batch descriptors"));
    if ((e = cudaMalloc((void **)&b->part_start, sizeof(int) * (n + 1))) != cudaSuccess ||
        (e = cudaMemcpy(b->part_start, ps.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(e, "batch particle list"));
    {
        std::vector<int *> ep(n);
        for (int k = 0; k < n; ++k) ep[k] = members[k]->err;
        void *q = nullptr;
        if ((e = cudaMalloc(&q, sizeof(int *) * n)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc batch errors"));
        b->err_ptrs = static_cast<int *const *>(q);
        if ((e = cudaMemcpy(q, ep.data(), sizeof(int *) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMalloc((void **)&b->err_out, sizeof(int) * n)) != cudaSuccess)
            return bail(cuda_fail(e, "batch error words"));
        b->err_host.assign(n, 0);
    }
    // order after every member's queued work, then build the launches
    for (cudaStream_t s : b->member_streams) {
        if ((e = cudaEventRecord(b->ev_in, s)) != cudaSuccess || (e = cudaStreamWaitEvent(b->stream, b->ev_in, 0)) != cudaSuccess)
            return bail(cuda_fail(e, "batch stream ordering"));
    }
    int rc;
    if ((rc = prepare_batch(b))) return bail(rc);
    *out = b;
    return DILBM_OK;
}

int dilbm_batch_step(dilbm_batch *b, long long nsteps) {
    const dilbm::TraceRange trace("dilbm_batch_step");
    if (!b || nsteps < 0) return fail(DILBM_ERR_INVALID_ARG, "bad batch or step count");
    if (nsteps == 0) return DILBM_OK;
    cudaError_t e;
    // a member stepped on its own since the descriptors were built: rebuild
    bool stale = false;
    for (size_t k = 0; k < b->members.size(); ++k)
        stale |= b->members[k]->cur != (b->cur0[k] ^ (int)(b->done & 1));
    for (cudaStream_t s : b->member_streams) {
        if ((e = cudaEventRecord(b->ev_in, s)) != cudaSuccess || (e = cudaStreamWaitEvent(b->stream, b->ev_in, 0)) != cudaSuccess)
            return cuda_fail(e, "batch stream ordering");
    }
    int rc;
    if (stale && (rc = prepare_batch(b))) return rc;
    long long left = nsteps;
    if (b->timing) {
        for (; left > 0; --left, ++b->done)
            if ((rc = batch_phase(b, (int)(b->done & 1)))) return rc;
    } else {
        if (b->done & 1) {                       // finish the pair in progress
            DILBM_CUDA(cudaGraphLaunch(b->g_single[1], b->stream));
            ++b->done;
            --left;
        }
        for (; left >= 2; left -= 2, b->done += 2) DILBM_CUDA(cudaGraphLaunch(b->g_pair, b->stream));
        if (left == 1) {
            DILBM_CUDA(cudaGraphLaunch(b->g_single[0], b->stream));
            ++b->done;
        }
        b->launches += nsteps * batch_launches_per_step(b);
    }
    for (size_t k = 0; k < b->members.size(); ++k) {
        dilbm_ctx *c = b->members[k];
        c->cur = b->cur0[k] ^ (int)(b->done & 1);
        c->fsum_steps += nsteps;
    }
    // members' own streams see the batch's work before anything queued later
    DILBM_CUDA(cudaEventRecord(b->ev_out, b->stream));
    for (cudaStream_t s : b->member_streams) DILBM_CUDA(cudaStreamWaitEvent(s, b->ev_out, 0));
    return DILBM_OK;
}

int dilbm_batch_sync(dilbm_batch *b, int *first_failed) {
    if (!b) return fail(DILBM_ERR_INVALID_ARG, "NULL batch");
    const int n = (int)b->members.size();
    gather_errors_kernel<<<(n + 255) / 256, 256, 0, b->stream>>>(b->err_ptrs, n, b->err_out);
    DILBM_CUDA(cudaGetLastError());
    b->launches += 1;
    DILBM_CUDA(cudaMemcpyAsync(b->err_host.data(), b->err_out, sizeof(int) * n, cudaMemcpyDeviceToHost, b->stream));
    DILBM_CUDA(cudaStreamSynchronize(b->stream));
    if (first_failed) *first_failed = -1;
    for (int k = 0; k < n; ++k) {
        dilbm_ctx *c = b->members[k];
        c->sticky |= b->err_host[k];
        if (c->sticky) {
            if (first_failed) *first_failed = k;
            return sticky_error(c->sticky);
        }
    }
    return DILBM_OK;
}

int dilbm_batch_errors(dilbm_batch *b, int *codes) {
    if (!b || !codes) return fail(DILBM_ERR_INVALID_ARG, "NULL argument");
    int first = -1;
    int rc = dilbm_batch_sync(b, &first);
    if (rc != DILBM_OK && first < 0) return rc;      // a CUDA error, not a member's
    for (size_t k = 0; k < b->members.size(); ++k) codes[k] = sticky_code(b->members[k]->sticky);
    return DILBM_OK;
}

int dilbm_batch_set_timing(dilbm_batch *b, int enable) {
    if (!b) return fail(DILBM_ERR_INVALID_ARG, "NULL batch");
    DILBM_CUDA(cudaStreamSynchronize(b->stream));
    b->timing = enable != 0;
    b->ev_used = 0;
    return DILBM_OK;
}

int dilbm_batch_sweep_time(dilbm_batch *b, double *ms_total, long long *launches) {
    if (!b || !ms_total || !launches) return fail(DILBM_ERR_INVALID_ARG, "NULL argument");
    DILBM_CUDA(cudaStreamSynchronize(b->stream));
    double total = 0.0;
    for (size_t k = 0; k + 1 < b->ev_used; k += 2) {
        float ms = 0.f;
        DILBM_CUDA(cudaEventElapsedTime(&ms, b->ev[k], b->ev[k + 1]));
        total += ms;
    }
    *ms_total = total;
    *launches = (long long)(b->ev_used / 2);
    return DILBM_OK;
}

long long dilbm_batch_launch_count(const dilbm_batch *b) { return b ? b->launches : -1; }

void dilbm_batch_destroy(dilbm_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->g_pair) cudaGraphExecDestroy(b->g_pair);
    for (int k = 0; k < 2; ++k) {
        if (b->g_single[k]) cudaGraphExecDestroy(b->g_single[k]);
        cudaFree(b->part_args[k]);
    }
    free_sweep_params(b);
    cudaFree(b->part_start);
    cudaFree((void *)b->err_ptrs);
    cudaFree(b->err_out);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"

// ---------------------------------------------------------------- autotuner
// Picks the sweep's launch shape (rows in flight per block, blocks per SM) by
// timing each candidate on the caller's own state.  Shapes do not change the
// arithmetic, so the choice is free to follow the clock.
namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, long long, long long>, SweepShape> g_tune;

// Candidate shapes, each with the warps it keeps resident per SM.
template <typename Occ>
int shape_candidates(Occ occupancy, std::vector<SweepShape> *out, std::vector<int> *warps_per_sm) {
    for (int w : SHAPE_WARPS) {
        int per_sm = 0;
        cudaError_t e = occupancy(SweepShape{w, 0}, &per_sm);
        if (e != cudaSuccess) return cuda_fail(e, "sweep occupancy");
        out->push_back(SweepShape{w, 0});
        warps_per_sm->push_back(w * per_sm);
        if (per_sm >= 2) {
            out->push_back(SweepShape{w, per_sm / 2});
            warps_per_sm->push_back(w * (per_sm / 2));
        }
    }
    return DILBM_OK;
}

// Time every candidate in TUNE_ROUNDS interleaved rounds of `reps` launches
// each (after one untimed launch) on `stream`; *best receives the candidate
// with the smallest median round time (interleaving spreads clock and
// neighbour noise over all candidates alike).  The full-occupancy shapes of
// the large sweeps differ by 1-2 %, so the median is taken over 7 rounds, and
// candidates within TUNE_TIE of the fastest count as tied: the one keeping the
// most warps resident per SM wins (a step runs the particle kernel between
// sweeps, and there the shape with more warps measured faster).
constexpr int TUNE_ROUNDS = 7;
constexpr float TUNE_TIE = 0.01f;

template <typename Launch>
int time_shapes(cudaStream_t stream, int reps, const std::vector<SweepShape> &cands, const std::vector<int> &warps_per_sm,
                Launch launch, SweepShape *best) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DILBM_CUDA(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    std::vector<float> ms(cands.size() * TUNE_ROUNDS, 0.f);
    for (int r = 0; r < TUNE_ROUNDS && e == cudaSuccess; ++r) {
        for (size_t k = 0; k < cands.size() && e == cudaSuccess; ++k) {
            e = launch(cands[k]);
            if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
            for (int q = 0; q < reps && e == cudaSuccess; ++q) e = launch(cands[k]);
            if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[k * TUNE_ROUNDS + r], e0, e1);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune launch");
    const bool log = std::getenv("DILBM_TUNE_LOG") != nullptr;
    std::vector<float> med(cands.size());
    float best_ms = 0.f;
    for (size_t k = 0; k < cands.size(); ++k) {
        float *m = &ms[k * TUNE_ROUNDS];
        std::sort(m, m + TUNE_ROUNDS);
        med[k] = m[TUNE_ROUNDS / 2];
        if (log)
            std::fprintf(stderr, "dilbm autotune: warps %d blocks/SM %d (%d warps per SM): median %.4f ms per %d launches\n",
                         cands[k].warps, cands[k].blocks_per_sm, warps_per_sm[k], med[k], reps);
        if (k == 0 || med[k] < best_ms) best_ms = med[k];
    }
    int pick = -1;
    for (size_t k = 0; k < cands.size(); ++k) {
        if (med[k] > best_ms * (1.0f + TUNE_TIE)) continue;
        if (pick < 0 || warps_per_sm[k] > warps_per_sm[pick] ||
            (warps_per_sm[k] == warps_per_sm[pick] && med[k] < med[pick]))
            pick = (int)k;
    }
    *best = cands[pick];
    return DILBM_OK;
}

bool tuned(const std::tuple<int, int, int, long long, long long> &key, SweepShape *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    *out = it->second;
    return true;
}

void remember(const std::tuple<int, int, int, long long, long long> &key, const SweepShape &sh) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = sh;
}

void report_shape(const SweepShape &sh, int *warps, int *blocks_per_sm) {
    if (warps) *warps = sh.warps;
    if (blocks_per_sm) *blocks_per_sm = sh.blocks_per_sm;
}

bool same_shape(const SweepShape &a, const SweepShape &b) {
    return a.warps == b.warps && a.blocks_per_sm == b.blocks_per_sm;
}

}  // namespace

extern "C" {

int dilbm_set_shape(dilbm_ctx *c, int warps, int blocks_per_sm) {
    const SweepShape sh{warps, blocks_per_sm};
    if (!c || !shape_valid(sh)) return fail(DILBM_ERR_INVALID_ARG, "warps must be 2, 4 or 8 and blocks_per_sm >= 0");
    if (c->method == DILBM_METHOD_PS && !same_shape(sh, SweepShape{}))
        return fail(DILBM_ERR_INVALID_ARG, "a PS-LBM context runs the sweep in the default shape (8 warps, 0)");
    if (!same_shape(sh, c->shape)) {
        DILBM_CUDA(cudaStreamSynchronize(c->stream));
        drop_graphs(c);
        c->shape = sh;
    }
    return DILBM_OK;
}

int dilbm_autotune(dilbm_ctx *c, int reps, int *warps, int *blocks_per_sm) {
    const dilbm::TraceRange trace("dilbm_autotune");
    if (!c) return fail(DILBM_ERR_INVALID_ARG, "NULL context");
    if (reps <= 0) reps = 10;
    if (c->method == DILBM_METHOD_PS) {         // one shape only: nothing to time
        report_shape(c->shape, warps, blocks_per_sm);
        return DILBM_OK;
    }
    const auto key = std::make_tuple(0, c->storage, has_edges(c) ? 1 : 0, (long long)c->L.nx, (long long)c->L.ny);
    SweepShape best = c->shape;
    if (!tuned(key, &best)) {
        std::vector<SweepShape> cands;
        std::vector<int> wps;
        int rc = shape_candidates([&](const SweepShape &sh, int *per_sm) { return step_sweep(c, sh, true, per_sm); },
                                  &cands, &wps);
        if (rc) return rc;
        // each launch sweeps the current state into the other buffer: what
        // the next step writes anyway
        rc = time_shapes(c->stream, reps, cands, wps, [&](const SweepShape &sh) { return step_sweep(c, sh); }, &best);
        c->launches += (long long)cands.size() * (reps + 1) * TUNE_ROUNDS;
        if (rc) return rc;
        remember(key, best);
    }
    report_shape(best, warps, blocks_per_sm);
    return dilbm_set_shape(c, best.warps, best.blocks_per_sm);
}

int dilbm_batch_set_shape(dilbm_batch *b, int warps, int blocks_per_sm) {
    const SweepShape sh{warps, blocks_per_sm};
    if (!b || !shape_valid(sh)) return fail(DILBM_ERR_INVALID_ARG, "warps must be 2, 4 or 8 and blocks_per_sm >= 0");
    if (same_shape(sh, b->shape)) return DILBM_OK;
    DILBM_CUDA(cudaStreamSynchronize(b->stream));
    b->shape = sh;
    return prepare_batch(b);     // re-capture the graphs in the new shape
}

int dilbm_batch_autotune(dilbm_batch *b, int reps, int *warps, int *blocks_per_sm) {
    const dilbm::TraceRange trace("dilbm_batch_autotune");
    if (!b) return fail(DILBM_ERR_INVALID_ARG, "NULL batch");
    if (reps <= 0) reps = 10;
    long long items = 0;
    for (const dilbm_ctx *c : b->members) items += (long long)c->L.ny * c->L.ntx;
    const auto key = std::make_tuple(1, b->storage, (int)b->members.size(), items, 0LL);
    SweepShape best = b->shape;
    if (!tuned(key, &best)) {
        cudaError_t e;
        // order after the members' queued work; bring the launches up to date
        for (cudaStream_t s : b->member_streams)
            if ((e = cudaEventRecord(b->ev_in, s)) != cudaSuccess || (e = cudaStreamWaitEvent(b->stream, b->ev_in, 0)) != cudaSuccess)
                return cuda_fail(e, "batch stream ordering");
        bool stale = false;
        for (size_t k = 0; k < b->members.size(); ++k)
            stale |= b->members[k]->cur != (b->cur0[k] ^ (int)(b->done & 1));
        int rc;
        if (stale && (rc = prepare_batch(b))) return rc;
        const int phase = (int)(b->done & 1);
        std::vector<SweepShape> cands;
        std::vector<int> wps;
        rc = shape_candidates(
            [&](const SweepShape &sh, int *per_sm) {
                switch (b->storage) {
                case DILBM_FP32: return launch_batch_sweep<float>(*static_cast<const BatchArgs<float> *>(b->sweep_params[0][0]), sh, 1, b->stream, true, per_sm);
                case DILBM_FP16_DEV: return launch_batch_sweep<__half>(*static_cast<const BatchArgs<__half> *>(b->sweep_params[0][0]), sh, 1, b->stream, true, per_sm);
                default: return launch_batch_sweep<__nv_bfloat16>(*static_cast<const BatchArgs<__nv_bfloat16> *>(b->sweep_params[0][0]), sh, 1, b->stream, true, per_sm);
                }
            },
            &cands, &wps);
        if (rc) return rc;
        rc = time_shapes(b->stream, reps, cands, wps, [&](const SweepShape &sh) { return batch_sweep(b, phase, sh); }, &best);
        b->launches += (long long)cands.size() * (reps + 1) * TUNE_ROUNDS * (long long)b->sweep_params[phase].size();
        if (rc) return rc;
        remember(key, best);
        if ((e = cudaEventRecord(b->ev_out, b->stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        for (cudaStream_t s : b->member_streams)
            if ((e = cudaStreamWaitEvent(s, b->ev_out, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    }
    report_shape(best, warps, blocks_per_sm);
    return dilbm_batch_set_shape(b, best.warps, best.blocks_per_sm);
}

}  // extern "C"
