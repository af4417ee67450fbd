// art_device.cuh -- device-side building blocks of the GB300 adaptive ray trace.
//
// * Double-float ("df") arithmetic: a value is an unevaluated sum hi + lo of two floats,
//   ~44 significant bits. Ray positions, face-crossing distances and split radii are held
//   this way so that a ray several hundred cells from its source still places its faces to
//   ~1e-11 cells, while every per-crossing operation stays on the FP32 pipes (FP64 throughput
//   on this part is a small fraction of FP32).
// * The ray-walk state and one crossing step of Sec. 2.1 (Kim et al. 2017): next face
//   crossing per axis measured from the source, segment length, attenuation
//   dL = L (1 - e^-dtau) with dtau = chi ds (Eq. e:RT2), deposit of sum dL/chi and sum dL n
//   (Eqs. e:Erad, e:Frad), retirement at tau > tau_max or on leaving the grid, split at
//   r_max(l).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace art {

constexpr int kNL = 20;                 // level slots (levels 0..13 used)
constexpr unsigned kFull = 0xffffffffu;
constexpr float kBig = 1.0e30f;         // "never": crossing distance of an axis with n_a = 0

// ---------------------------------------------------------------------------------------
// double-float arithmetic
// ---------------------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df df_quick(float a, float b)  // requires |a| >= |b|
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b)
{
    df s = df_two_sum(a.hi, b.hi);
    return df_quick(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_mul(df a, df b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_quick(p, e);
}
__device__ __forceinline__ df df_div(df a, df b)
{
    float q1 = __fdiv_rn(a.hi, b.hi);
    df r = df_add(a, df_neg(df_mul({q1, 0.f}, b)));
    float q2 = __fdiv_rn(r.hi, b.hi);
    return df_quick(q1, q2);
}
// a <= b for normalised df values (lexicographic on hi, lo)
__device__ __forceinline__ bool df_le(df a, df b)
{
    return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}
// a - b rounded to float; exact enough when a and b are close (Sterbenz on hi)
__device__ __forceinline__ float df_diff(df a, df b)
{
    return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
}

// ---------------------------------------------------------------------------------------
// shared data layouts
// ---------------------------------------------------------------------------------------

// Per source: position in cell units (df split over two float4) + base-ray luminosity and
// the source's l_max.
struct SrcDev {
    float4 hi;  // u_x, u_y, u_z (hi parts), L / N_ray(l0)
    float4 lo;  // u_x, u_y, u_z (lo parts), l_max (int bits)
};

// Per level constants of a trace.
struct LevelInfo {
    df r0;              // start radius of level-l rays (r_max(l-1), 0 at l0), cell units
    df rmax;            // split radius r_max(l), cell units
    const float4* dir_hi;  // direction table of level l: hi parts (w unused)
    const float4* dir_lo;  //                              lo parts
    unsigned long long destroy_w;  // 4^(l_max_global - l)
};

// SoA ray buffer of one level: source index, nested pixel, entering L and tau.
struct RayBuf {
    unsigned* src;
    unsigned* pix;
    float* L;
    float* tau;
    // adjoint extras (NULL in forward traces)
    unsigned* parent;   // slot of the parent in the level above
    float* own;         // weighted sum over the ray's own segments (pass 1)
    float* sub;         // weighted sum over the ray's descendants (filled by the children)
    unsigned long long cap;
};

// Per-thread tallies, reduced per block at kernel exit.
struct Tally {
    double escaped, dropped, absorbed;
    unsigned long long crossings, destroy;
};

// Device-resident counters of one trace.
struct DevStats {
    unsigned long long crossings, destroy, rays_total;
    unsigned long long rays_per_level[kNL];
    double escaped, dropped, absorbed;
    int level_reached;
    int error;
};

// Scheduler state of the persistent trace and of the plain per-level launches.
struct Sched {
    unsigned long long count[kNL];   // rays held in the level buffer (a stack, top = count)
    unsigned long long cursor[kNL];  // next ray of the current phase / launch
    unsigned long long phase_begin, phase_end;
    unsigned long long chunk_begin[kNL], chunk_end[kNL];  // adjoint: expanded range per level
    int chunk_state[kNL];
    int phase_level, phase_kind, done, pad;
    unsigned bar_count, bar_gen;
};

// Everything the trace kernels read.
struct TraceArgs {
    int nx, ny, nz;
    int level0, lmax_glob;
    int chunk;
    float tau_max;
    const float* chi;        // opacity per cell times dx (per cell length)
    const float* chiH;       // neutral-H part of chi (adjoint only)
    const float* w;          // adjoint weights per cell
    float* grad;             // adjoint output per cell
    double* dL;              // adjoint output per source
    float4* acc;             // per-cell accumulator (sum L ds phi, sum dL n)
    const SrcDev* src;
    const LevelInfo* levels;
    RayBuf buf[kNL];
    Sched* sched;
    DevStats* stats;
    long long wait_ns;       // bound of a grid-barrier wait (<0: give up at once)
    float gscale;            // adjoint: sigma_H * dx / dV (gamma per unit G)
};

enum : int { EV_NONE = 0, EV_EXIT = 1, EV_DROP = 2, EV_SPLIT = 3 };

// ---------------------------------------------------------------------------------------
// ray walk
// ---------------------------------------------------------------------------------------
struct Walk {
    df t[3];      // distance from the source to the next face on each axis
    df dt[3];     // distance between consecutive faces on each axis
    df tc;        // distance of the current position
    df te;        // split radius, or kBig for rays that never split
    int idx;      // linear index of the current cell
    int rem[3];   // cells left on each axis before the ray leaves the grid
    int stride[3];
    float n[3];   // direction (hi parts) for momentum deposits
    float L, tau;
    float chi;    // opacity of the current cell (prefetched)
};

// Sets up the walk of a ray of level l with direction n (df) from source position u (df)
// starting at radius r0. Returns false if the start point lies outside the grid.
__device__ __forceinline__ bool walk_start(Walk& W, const TraceArgs& A, const df u[3],
                                           const df n[3], df r0, df te)
{
    const int N[3] = {A.nx, A.ny, A.nz};
    int c[3];
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        df p = (r0.hi == 0.f) ? u[a] : df_add(u[a], df_mul(r0, n[a]));
        float f = floorf(p.hi);
        int ci = (int)f;
        if (p.hi == f && (p.lo < 0.f || (p.lo == 0.f && n[a].hi < 0.f))) ci -= 1;
        c[a] = ci;
        inside = inside && ci >= 0 && ci < N[a];
        W.n[a] = n[a].hi;
        if (n[a].hi > 0.f) {
            W.rem[a] = N[a] - 1 - ci;
            W.t[a] = df_div(df_add({(float)(ci + 1), 0.f}, df_neg(u[a])), n[a]);
            W.dt[a] = df_div({1.f, 0.f}, n[a]);
        } else if (n[a].hi < 0.f) {
            W.rem[a] = ci;
            W.t[a] = df_div(df_add({(float)ci, 0.f}, df_neg(u[a])), n[a]);
            W.dt[a] = df_div({1.f, 0.f}, df_neg(n[a]));
        } else {
            W.rem[a] = 1 << 30;
            W.t[a] = {kBig, 0.f};
            W.dt[a] = {0.f, 0.f};
        }
    }
    W.stride[0] = W.n[0] > 0.f ? 1 : -1;
    W.stride[1] = W.n[1] > 0.f ? A.nx : -A.nx;
    W.stride[2] = W.n[2] > 0.f ? A.nx * A.ny : -(A.nx * A.ny);
    W.tc = r0;
    W.te = te;
    W.idx = inside ? c[0] + A.nx * (c[1] + A.ny * c[2]) : 0;
    return inside;
}

// Outcome of one crossing step: the deposit to make (cell < 0: none) and the event.
struct StepOut {
    int cell;
    float ds;     // segment length (cell units), > 0 when cell >= 0
    float dtau;
    float Lin;
    float G;      // L_in ds phi(dtau)
    float dL;
    int ev;
};

__device__ __forceinline__ float phi_of(float dtau, float em)
{
    // (1 - e^-x)/x from em = expm1(-x); series below 1e-4
    return dtau > 1e-4f ? __fdividef(-em, dtau)
                        : fmaf(dtau, fmaf(dtau, 1.f / 6.f, -0.5f), 1.f);
}

// One step of the walk: the segment from tc to the next face or the split radius.
template <bool kCountOnly>
__device__ __forceinline__ StepOut walk_step(Walk& W, const float* __restrict__ chi_arr,
                                             float tau_max)
{
    StepOut o;
    // earliest face crossing (lexicographic on the normalised df values)
    bool l01 = df_le(W.t[0], W.t[1]);
    df t01 = l01 ? W.t[0] : W.t[1];
    bool l2 = df_le(t01, W.t[2]);
    df tm = l2 ? t01 : W.t[2];
    bool split = df_le(W.te, tm);
    df tend = split ? W.te : tm;
    o.ds = df_diff(tend, W.tc);
    // axes that cross together with the earliest one (relative tie 1e-12)
    const float tol = 1e-12f * tm.hi;
    int mask = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (df_diff(W.t[a], tm) <= tol) mask |= 1 << a;
    // next cell, and prefetch of its opacity
    int nidx = W.idx;
    bool out = false;
    if (!split) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (mask & (1 << a)) {
                nidx += W.stride[a];
                out = out || (W.rem[a] == 0);
            }
    }
    float nchi = 0.f;
    if (!split && !out) nchi = __ldg(chi_arr + nidx);
    // deposit in the current cell
    o.cell = -1;
    o.ev = EV_NONE;
    o.Lin = W.L;
    o.G = 0.f;
    o.dL = 0.f;
    o.dtau = 0.f;
    if (o.ds > 0.f) {
        o.cell = W.idx;
        float dtau = W.chi * o.ds;
        o.dtau = dtau;
        if (!kCountOnly) {
            float em = expm1f(-dtau);
            o.dL = -W.L * em;
            o.G = W.L * o.ds * phi_of(dtau, em);
            W.L = W.L - o.dL;
        }
        W.tau += dtau;
        if (W.tau > tau_max) o.ev = EV_DROP;
    }
    if (o.ev == EV_NONE) {
        if (split) {
            o.ev = EV_SPLIT;
        } else if (out) {
            o.ev = EV_EXIT;
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (mask & (1 << a)) {
                    W.rem[a] -= 1;
                    W.t[a] = df_add(W.t[a], W.dt[a]);
                }
            W.tc = tm;
            W.idx = nidx;
            W.chi = nchi;
        }
    }
    return o;
}

// Merges deposits of adjacent lanes that hit the same cell (runs of equal cell index in
// lane order), then issues one 16-byte vector reduction per run head. Warp-uniform.
__device__ __forceinline__ void deposit_warp(float4* __restrict__ acc, int cell, float4 v)
{
    const unsigned lane = threadIdx.x & 31u;
    int prev = __shfl_up_sync(kFull, cell, 1);
    bool dup = lane > 0 && cell >= 0 && prev == cell;
    unsigned dups = __ballot_sync(kFull, dup);
    if (dups) {
        unsigned heads = ~dups;
        unsigned after = heads & ~((2u << lane) - 1u);
        if (lane == 31) after = 0;
        int run_end = after ? __ffs(after) - 1 : 32;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            float ox = __shfl_down_sync(kFull, v.x, off);
            float oy = __shfl_down_sync(kFull, v.y, off);
            float oz = __shfl_down_sync(kFull, v.z, off);
            float ow = __shfl_down_sync(kFull, v.w, off);
            if ((int)lane + off < run_end) {
                v.x += ox; v.y += oy; v.z += oz; v.w += ow;
            }
        }
        if (dup) cell = -1;
    }
    if (cell >= 0) {
        float* p = reinterpret_cast<float*>(acc + cell);
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x),
                     "f"(v.y), "f"(v.z), "f"(v.w)
                     : "memory");
    }
}

}  // namespace art
