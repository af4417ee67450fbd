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
    const float4* dir;     // direction table of level l: 3 float4 per pixel holding
                           // n (hi, lo) and 1/n (hi, lo) per axis
    unsigned long long destroy_w;  // 4^(l_max_global - l)
};

// SoA ray buffer of one level: source index, nested pixel, entering L and tau.
struct RayBuf {
    unsigned* src;
    unsigned* pix;
    float* L;
    float* tau;
    float* Ln;          // two-bin traces: entering L and tau of the non-ionizing bin
    float* taun;
    // adjoint extras (NULL in forward traces)
    unsigned* parent;   // slot of the parent in the level above
    float2* own;        // weighted sum over the ray's own segments (pass 1), double-float
    float* sub;         // weighted sum over the ray's descendants (added by the children)
    unsigned* pending;  // children of a split ray still to finish
    unsigned long long cap;
};

// Per-thread tallies, reduced per block at kernel exit.
struct Tally {
    double escaped, dropped;
    unsigned long long crossings, destroy;
    double escaped_n, dropped_n;  // non-ionizing bin of two-bin traces
};

// Device-resident counters of one trace.
struct DevStats {
    unsigned long long crossings, destroy, rays_total;
    unsigned long long rays_per_level[kNL];
    double escaped, dropped;
    double escaped_n, dropped_n;
    int level_reached;
    int error;
};

// Scheduler state of the persistent trace and of the plain per-level launches.
struct Sched {
    unsigned long long count[kNL];   // rays held in the level buffer (a stack, top = count)
    unsigned long long cursor[kNL];  // next ray of the current phase / launch
    unsigned long long phase_begin, phase_end;
    int phase_level, phase_kind, done, pad;
    unsigned bar_count, bar_gen;
};

// Everything the trace kernels read.
struct CellF;
struct CellW;

struct TraceArgs {
    int nx, ny, nz;
    int level0, lmax_glob;
    int chunk;
    float tau_max;
    const float* chi;        // opacity per cell times dx (per cell length), padded layout
    const float2* chi2;      // two-bin traces: {chi_i, chi_n} per cell length, padded
    const float* srcLn;      // two-bin traces: base-ray non-ionizing luminosity per source
    const float4* rec;       // adjoint: per cell {chi, chi_H, w, 0}
    const float* w;          // adjoint weights per cell
    float* grad;             // adjoint gradient per cell (padded scratch)
    double* dL;              // adjoint output per source
    float4* acc;             // per-cell accumulator (sum L ds phi, sum dL n), padded
    const SrcDev* src;
    const LevelInfo* levels;
    RayBuf buf[kNL];
    Sched* sched;
    DevStats* stats;
    long long wait_ns;       // bound of a grid-barrier wait (<0: give up at once)
    float gscale;            // adjoint: sigma_H * dx / dV (gamma per unit G)
    const float* srcL;       // adjoint: source luminosities (gradients scale with them)
    const CellF* recf;       // adjoint with a force term: per cell {chi, chi_H, w, 0}, {v, 0}
    const CellW* recw;       // adjoint without dust and force term: per cell {chi, w}
    df dmax;                 // d_max cutoff in cell units (kernels built for a cutoff only)
    float fscale;            // adjoint: force per unit momentum (1 / dV)
};

enum : int { EV_NONE = 0, EV_EXIT = 1, EV_DROP = 2, EV_SPLIT = 3 };

// ---------------------------------------------------------------------------------------
// ray walk
// ---------------------------------------------------------------------------------------
// Per-cell record gathered at every step: the opacity alone (forward), or
// {opacity, its neutral-H part, loss weight, unused} (adjoint).
__device__ __forceinline__ float chi_of(const float& c) { return c; }
__device__ __forceinline__ float chi_of(const float4& c) { return c.x; }
__device__ __forceinline__ float chi_of(const float2& c) { return c.x; }
// A cell record of two floats marks a two-bin trace: {chi_i, chi_n}.
template <class Cell> struct TwoBin { static constexpr bool value = false; };
template <> struct TwoBin<float2> { static constexpr bool value = true; };
__device__ __forceinline__ float load_cell(const float* p) { return __ldg(p); }
__device__ __forceinline__ float4 load_cell(const float4* p) { return __ldg(p); }
__device__ __forceinline__ float2 load_cell(const float2* p) { return __ldg(p); }
template <class Cell> __device__ __forceinline__ Cell cell_zero();
template <> __device__ __forceinline__ float cell_zero<float>() { return 0.f; }
template <> __device__ __forceinline__ float4 cell_zero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ float2 cell_zero<float2>() { return make_float2(0.f, 0.f); }
// Cell record of a reverse sweep whose loss has a force term: {chi, chi_H, w, 0} and the
// force weight {v_x, v_y, v_z, 0} (32 bytes, two 16-byte gathers per step).
struct CellF {
    float4 a, b;
};
__device__ __forceinline__ float chi_of(const CellF& c) { return c.a.x; }
__device__ __forceinline__ CellF load_cell(const CellF* p) { return {__ldg(&p->a), __ldg(&p->b)}; }
// Cell record of a reverse sweep without dust and without a force term: {chi, w} (8 bytes).
// Without dust the neutral-H opacity is chi itself (both are float(n_H0 sigma_H dx)).
struct __align__(8) CellW {
    float chi, w;
};
__device__ __forceinline__ float chi_of(const CellW& c) { return c.chi; }
__device__ __forceinline__ CellW load_cell(const CellW* p)
{
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
template <> __device__ __forceinline__ CellW cell_zero<CellW>() { return {0.f, 0.f}; }
template <> __device__ __forceinline__ CellF cell_zero<CellF>()
{
    return {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
}

template <class Cell>
struct WalkT {
    df t[3];      // distance from the source to the next face on each axis
    df d[3];      // distance between consecutive faces on each axis (1/|n_a|)
    df tc;        // distance of the current position
    int idx;      // index of the current cell in the padded layout (sentinel ring around
                  // the grid, see pad_index)
    int ss[3];    // signed index step of a crossing on each axis
    float n[3];   // direction (hi parts) for momentum deposits
    float L, tau;
    float Lc;        // photon ledger: the rounding error of this walk's L updates (see
                     // walk_step); tallied with the ray, never used for deposits
    float Ln, taun;  // non-ionizing bin (two-bin traces only)
    float Lnc;       // the same compensation for Ln
    Cell cell;    // record of the current cell (prefetched)
};
using Walk = WalkT<float>;

// Cell records are stored with a ring of sentinel cells around the nx*ny*nz grid (opacity
// < 0): cell (i, j, k) sits at (i + 1) + (nx + 2) ((j + 1) + (ny + 2) (k + 1)). A ray leaves
// the grid when the cell it steps into is a sentinel, so the walk keeps no per-axis count of
// cells left, and the cell after any crossing from inside the grid is a valid address.
__host__ __device__ __forceinline__ long long pad_index(long long i, long long j, long long k,
                                                        int nx, int ny)
{
    return (i + 1) + (long long)(nx + 2) * ((j + 1) + (long long)(ny + 2) * (k + 1));
}
constexpr float kSentinel = -1.0f;

// Coordinates of padded cell q (see pad_index; padded grids hold fewer than 2^31 cells):
// false for the sentinel ring, else the cell's index in the caller's nx*ny*nz layout.
__device__ __forceinline__ bool unpad(unsigned q, int nx, int ny, int nz, unsigned& i)
{
    const unsigned px = (unsigned)nx + 2u, py = (unsigned)ny + 2u;
    const unsigned r = q / px;
    const int X = (int)(q - r * px) - 1;
    const int Y = (int)(r % py) - 1;
    const int Z = (int)(r / py) - 1;
    i = (unsigned)X + (unsigned)nx * ((unsigned)Y + (unsigned)ny * (unsigned)Z);
    return X >= 0 && X < nx && Y >= 0 && Y < ny && Z >= 0 && Z < nz;
}

// Padded index of cell i of the caller's nx*ny*nz layout.
__device__ __forceinline__ unsigned pad_of(unsigned i, int nx, int ny)
{
    const unsigned r = i / (unsigned)nx, x = i - r * (unsigned)nx;
    return (unsigned)pad_index(x, r % (unsigned)ny, r / (unsigned)ny, nx, ny);
}

// Sets up the walk of a ray with direction n and reciprocal inv (df, from the direction
// table) from source position u (df) starting at radius r0. Returns false if the start
// point lies outside the grid.
template <class Cell>
__device__ __forceinline__ bool walk_start(WalkT<Cell>& W, int nx, int ny, int nz, const df u[3],
                                           const df n[3], const df inv[3], df r0)
{
    const int N[3] = {nx, ny, nz};
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
        if (n[a].hi != 0.f) {
            const bool up = n[a].hi > 0.f;
            const int stride = a == 0 ? 1 : (a == 1 ? nx + 2 : (nx + 2) * (ny + 2));
            W.ss[a] = up ? stride : -stride;
            const df off = df_add({(float)(up ? ci + 1 : ci), 0.f}, df_neg(u[a]));
            W.t[a] = df_mul(off, inv[a]);
            W.d[a] = up ? inv[a] : df_neg(inv[a]);
        } else {
            W.ss[a] = 0;
            W.t[a] = {kBig, 0.f};
            W.d[a] = {0.f, 0.f};
        }
    }
    W.tc = r0;
    W.idx = inside ? (int)pad_index(c[0], c[1], c[2], nx, ny) : 0;
    return inside;
}

// Outcome of one crossing step: the deposit to make (in cell, when seg) and the event.
struct StepOut {
    int cell;     // the cell the segment lies in (padded layout)
    bool seg;     // the segment has positive length: deposit and count it
    bool end;     // the ray ends with this step (ev != EV_NONE)
    float ds;     // segment length (cell units), > 0 when seg
    float dtau;
    float Lin;
    float G;      // L_in ds phi(dtau)
    float dL;     // L_in (1 - e^-dtau)
    float phi;    // (1 - e^-dtau)/dtau
    float dphi;   // d phi / d dtau (filled by walk_step<kCountOnly, true> only)
    float dLn;    // two-bin traces: loss of the non-ionizing bin (chi_n = n_H sigma_d)
    int ev;
};

// (1 - e^-x)/x for x >= 0. Below 1 as e^{-x/2} sinh(x/2)/(x/2), the even series of
// sinh(y)/y to y^8 (truncation < 3e-11 for y < 1/2, no cancellation); above 1 as
// (1 - e^{-x})/x with e^{-x} = (e^{-x/2})^2. One exponential serves both branches, which are
// evaluated and selected, so lanes never diverge here.
__device__ __forceinline__ float phi_of(float x)
{
    const float y = 0.5f * x;
    const float E = __expf(-y);
    const float y2 = y * y;
    float S = fmaf(y2, 1.f / 362880.f, 1.f / 5040.f);
    S = fmaf(S, y2, 1.f / 120.f);
    S = fmaf(S, y2, 1.f / 6.f);
    S = fmaf(S, y2, 1.f);
    const float small = E * S;
    const float large = __fdividef(fmaf(-E, E, 1.f), fmaxf(x, 1.f));
    return x < 1.f ? small : large;
}

// phi(x) and phi'(x) from the same exponential (the reverse sweep needs both). Below 1, with
// y = x/2, E = e^{-y} and S = sinh(y)/y: phi = E S and phi' = E (S'(y) - S) / 2, S' to y^7
// (S' - S stays near -1, so nothing cancels); above 1, phi' = (e^{-x} - phi)/x.
__device__ __forceinline__ float phi_dphi(float x, float& dphi)
{
    const float y = 0.5f * x;
    const float E = __expf(-y);
    const float y2 = y * y;
    float S = fmaf(y2, 1.f / 362880.f, 1.f / 5040.f);
    S = fmaf(S, y2, 1.f / 120.f);
    S = fmaf(S, y2, 1.f / 6.f);
    S = fmaf(S, y2, 1.f);
    float Sp = fmaf(y2, 1.f / 45360.f, 1.f / 840.f);
    Sp = fmaf(Sp, y2, 1.f / 30.f);
    Sp = fmaf(Sp, y2, 1.f / 3.f);
    Sp *= y;
    const float r = __fdividef(1.f, fmaxf(x, 1.f));
    const float E2 = E * E;
    const float large = (1.f - E2) * r;
    const bool sm = x < 1.f;
    dphi = sm ? 0.5f * E * (Sp - S) : (E2 - large) * r;
    return sm ? E * S : large;
}

__device__ __forceinline__ df df_sel(bool c, df a, df b) { return {c ? a.hi : b.hi, c ? a.lo : b.lo}; }

// One step of the walk: the segment from tc to the next face or to the split radius rmax
// (when the ray splits at all). The common case (one axis crossing) runs without branches;
// faces crossed together (ties) take a short side path. When the step ends the ray (event
// other than EV_NONE) the walk state other than L and tau is left unspecified.
template <bool kCountOnly, bool kDphi = false, class Cell>
__device__ __forceinline__ StepOut walk_step(WalkT<Cell>& W, bool splits, df rmax,
                                             const Cell* __restrict__ cells, float tau_max)
{
    StepOut o;
    // A step that starts in a sentinel cell ends the ray: it left the grid with the crossing
    // of the previous step (whose segment was deposited then); nothing is deposited now.
    const bool out = chi_of(W.cell) < 0.f;
    // Earliest face crossing, decided on the hi parts: for normalised df values |lo| is at
    // most half an ulp of hi, so distinct hi parts order the values exactly. Equal hi parts
    // (exact ties, near ties, a face at the split radius) take the exact double-float path
    // below. Two values within the 1e-12 tie tolerance can still have distinct hi parts when
    // they straddle a rounding boundary of hi; the walk then crosses the two faces in two
    // steps with a segment far below the 1e-5-cell near-tie threshold between them, a ray
    // the oracle flags as near-tie.
    const float h0 = W.t[0].hi, h1 = W.t[1].hi, h2 = W.t[2].hi;
    const bool c01 = h0 < h1;
    const float h01 = c01 ? h0 : h1;
    const bool c2 = h01 < h2;
    bool p0 = c2 && c01, p1 = c2 && !c01, p2 = !c2;  // the earliest axis
    const float hm = c2 ? h01 : h2;
    df tm = {hm, p2 ? W.t[2].lo : (c01 ? W.t[0].lo : W.t[1].lo)};
    bool split = splits && rmax.hi < hm;
    // next cell, for the usual single-axis crossing
    int nidx = W.idx + (p2 ? W.ss[2] : (c01 ? W.ss[0] : W.ss[1]));
    // the second-earliest hi part: a tie with the earliest face, or the split radius at the
    // earliest face, needs the exact comparison (axes parallel to the grid sit at kBig and
    // tie only with each other, never with the earliest face)
    const float h2nd = c2 ? fminf(c01 ? h1 : h0, h2) : h01;
    if (h2nd == hm || (splits && rmax.hi == hm)) {
        const bool e01 = df_le(W.t[0], W.t[1]);
        tm = df_sel(e01, W.t[0], W.t[1]);
        int a = e01 ? 0 : 1;
        if (!df_le(tm, W.t[2])) {
            tm = W.t[2];
            a = 2;
        }
        p0 = a == 0;
        p1 = a == 1;
        p2 = a == 2;
        split = splits && df_le(rmax, tm);
        // axes crossing together with the earliest one (relative tie 1e-12): a diagonal step
        const float tol = 1e-12f * tm.hi;
        const bool m0 = df_diff(W.t[0], tm) <= tol;
        const bool m1 = df_diff(W.t[1], tm) <= tol;
        const bool m2 = df_diff(W.t[2], tm) <= tol;
        nidx = W.idx + (m0 ? W.ss[0] : 0) + (m1 ? W.ss[1] : 0) + (m2 ? W.ss[2] : 0);
        // tied axes other than a advance here; axis a advances with the common path below
        if (m0 && a != 0) W.t[0] = df_add(W.t[0], W.d[0]);
        if (m1 && a != 1) W.t[1] = df_add(W.t[1], W.d[1]);
        if (m2 && a != 2) W.t[2] = df_add(W.t[2], W.d[2]);
    }
    o.ds = df_diff(split ? rmax : tm, W.tc);
    // prefetch of the next cell: from a cell inside the grid every crossing (also a diagonal
    // one) lands inside the padded layout
    const Cell ncell = out ? cell_zero<Cell>() : load_cell(cells + nidx);
    // deposit in the current cell (segments of length <= 0 deposit nothing)
    const bool seg = !out && o.ds > 0.f;
    const float ds = seg ? o.ds : 0.f;
    const float x = chi_of(W.cell) * ds;
    o.cell = W.idx;
    o.seg = seg;
    o.Lin = W.L;
    o.dtau = x;
    if (!kCountOnly) {
        float ph;
        if constexpr (kDphi) ph = phi_dphi(x, o.dphi);
        else ph = phi_of(x);
        o.phi = ph;
        o.G = W.L * ds * ph;
        o.dL = W.L * x * ph;
        // L - dL, and its rounding error (Fast2Sum, dL <= L) kept for the photon ledger:
        // where a cell is nearly transparent dL falls below half an ulp of L, so the
        // deposited dL never leaves L. The deposits keep using L itself, whose relative
        // accuracy survives strong attenuation (L + Lc carries the absolute error of all
        // deposits instead); only the tallies of retired rays take L + Lc.
        const float Lnew = __fsub_rn(W.L, o.dL);
        W.Lc = __fadd_rn(W.Lc, __fsub_rn(__fsub_rn(W.L, Lnew), o.dL));
        W.L = Lnew;
    } else {
        o.phi = 1.f;
        o.G = 0.f;
        o.dL = 0.f;
    }
    W.tau += x;
    bool drop;
    if constexpr (TwoBin<Cell>::value) {
        // second bin on the same ray; the packet is used up once its dust-only depth (never
        // the larger one) passes tau_max
        const float xn = W.cell.y * ds;
        o.dLn = W.Ln * xn * phi_of(xn);
        const float Lnnew = __fsub_rn(W.Ln, o.dLn);
        W.Lnc = __fadd_rn(W.Lnc, __fsub_rn(__fsub_rn(W.Ln, Lnnew), o.dLn));
        W.Ln = Lnnew;
        W.taun += xn;
        drop = seg && W.taun > tau_max;
    } else {
        o.dLn = 0.f;
        drop = seg && W.tau > tau_max;
    }
    o.end = out || drop || split;
    o.ev = out ? EV_EXIT : (drop ? EV_DROP : (split ? EV_SPLIT : EV_NONE));
    // advance: the earliest axis by select, further tied axes on the side path
    const df dsel = {p0 ? W.d[0].hi : (p1 ? W.d[1].hi : W.d[2].hi),
                     p0 ? W.d[0].lo : (p1 ? W.d[1].lo : W.d[2].lo)};
    const df tn = df_add(tm, dsel);
    W.t[0] = df_sel(p0, tn, W.t[0]);
    W.t[1] = df_sel(p1, tn, W.t[1]);
    W.t[2] = df_sel(p2, tn, W.t[2]);
    W.tc = tm;
    W.idx = nidx;
    W.cell = ncell;
    return o;
}

// Merges the deposits of lanes that hit the same cell (runs of equal cell index in lane
// order) and issues one reduction per run. Used only for the first segment of base-level
// rays, which all start in their source's cell: at l0 = 8 that is 786,432 deposits into one
// cell per source, whose FP32 sum the merge keeps accurate. Warp-uniform.
__device__ __forceinline__ void red_v4(float4* q, float4 v)
{
    float* p = reinterpret_cast<float*>(q);
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ void deposit_merged(float4* __restrict__ acc, int cell, float4 v)
{
    const unsigned lane = threadIdx.x & 31u;
    const int prev = __shfl_up_sync(kFull, cell, 1);
    const bool dup = lane > 0 && cell >= 0 && prev == cell;
    const unsigned dups = __ballot_sync(kFull, dup);
    const unsigned after = lane == 31 ? 0u : ~dups & ~((2u << lane) - 1u);
    const int run_end = after ? __ffs(after) - 1 : 32;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float ox = __shfl_down_sync(kFull, v.x, off);
        const float oy = __shfl_down_sync(kFull, v.y, off);
        const float oz = __shfl_down_sync(kFull, v.z, off);
        const float ow = __shfl_down_sync(kFull, v.w, off);
        if ((int)lane + off < run_end) {
            v.x += ox; v.y += oy; v.z += oz; v.w += ow;
        }
    }
    if (cell >= 0 && !dup) red_v4(acc + cell, v);
}

// One 16-byte vector reduction (G, dL n) into the accumulator of `cell` (none if < 0).
// Merging equal cells across lanes first was measured slower than letting L2 combine them.
__device__ __forceinline__ void deposit(float4* __restrict__ acc, int cell, float4 v)
{
    if (cell >= 0) red_v4(acc + cell, v);
}
__device__ __forceinline__ void deposit_if(float4* __restrict__ acc, bool dep, int cell, float4 v)
{
    if (dep) red_v4(acc + cell, v);
}

// ---------------------------------------------------------------------------------------
// helpers shared by the forward and backward kernels
// ---------------------------------------------------------------------------------------
// Per-warp tallies live in shared memory (one Tally per warp, updated with shared atomics
// when a ray ends), so they cost no registers in the walk loop.
__device__ __forceinline__ Tally* tally_slots()
{
    __shared__ Tally s_t[32];
    return s_t;
}

__device__ __forceinline__ void tally_init()
{
    Tally* t = tally_slots();
    if (threadIdx.x < 32) t[threadIdx.x] = Tally{0.0, 0.0, 0ull, 0ull, 0.0, 0.0};
    __syncthreads();
}

// Adds a lane count of crossings to its warp's tally.
__device__ __forceinline__ void tally_crossings(Tally& T, unsigned n)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) n += __shfl_down_sync(kFull, n, off);
    if ((threadIdx.x & 31u) == 0 && n > 0) atomicAdd(&T.crossings, (unsigned long long)n);
}

__device__ __forceinline__ void tally_flush(DevStats* st)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const Tally* t = tally_slots();
        Tally s = {0.0, 0.0, 0ull, 0ull, 0.0, 0.0};
        for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w) {
            s.escaped += t[w].escaped;
            s.dropped += t[w].dropped;
            s.escaped_n += t[w].escaped_n;
            s.dropped_n += t[w].dropped_n;
            s.crossings += t[w].crossings;
            s.destroy += t[w].destroy;
        }
        atomicAdd(&st->escaped, s.escaped);
        atomicAdd(&st->dropped, s.dropped);
        if (s.escaped_n != 0.0) atomicAdd(&st->escaped_n, s.escaped_n);
        if (s.dropped_n != 0.0) atomicAdd(&st->dropped_n, s.dropped_n);
        atomicAdd(&st->crossings, s.crossings);
        atomicAdd(&st->destroy, s.destroy);
    }
}

// Slot value of a ray buffer entry that holds no ray: the children slots of a parent that
// did not split (each parent owns four consecutive child slots, so fronts keep pixel order).
constexpr unsigned kHole = 0xffffffffu;

// With a d_max cutoff: where a ray of a level with split radius rmax ends, and whether it
// splits there. A ray that can split ends at min(rmax, d_max); at equal radii the cut wins.
__device__ __forceinline__ df end_radius(bool splits, df rmax, df dmax)
{
    return (splits && !df_le(dmax, rmax)) ? rmax : dmax;
}
__device__ __forceinline__ bool splits_at_end(bool splits, df rmax, df dmax)
{
    return splits && !df_le(dmax, rmax);
}

// Starts the walk of ray i of level l: loads its record, its source and its direction
// entry. Returns 1 if the ray starts inside the grid, 0 if it starts outside (it escapes at
// once), -1 if slot i holds no ray. L0 receives its entering L.
template <class Cell>
__device__ __forceinline__ int ray_begin(const TraceArgs& A, const LevelInfo& LV, const RayBuf& B,
                                         int l, unsigned long long i, WalkT<Cell>& W,
                                         const Cell* cells, unsigned& s, unsigned& p, float& L0,
                                         bool& splits)
{
    s = __ldcg(B.src + i);
    if (s == kHole) return -1;
    p = __ldcg(B.pix + i);
    const float4 sh = __ldg(&A.src[s].hi);
    const float4 sl = __ldg(&A.src[s].lo);
    L0 = (l == A.level0) ? sh.w : __ldcg(B.L + i);
    const float tau0 = (l == A.level0) ? 0.f : __ldcg(B.tau + i);
    splits = l < __float_as_int(sl.w);
    const float4 e0 = __ldg(LV.dir + 3ull * p);
    const float4 e1 = __ldg(LV.dir + 3ull * p + 1);
    const float4 e2 = __ldg(LV.dir + 3ull * p + 2);
    const df u[3] = {{sh.x, sl.x}, {sh.y, sl.y}, {sh.z, sl.z}};
    const df n[3] = {{e0.x, e0.w}, {e0.y, e1.x}, {e0.z, e1.y}};
    const df inv[3] = {{e1.z, e2.y}, {e1.w, e2.z}, {e2.x, e2.w}};
    const bool inside = walk_start(W, A.nx, A.ny, A.nz, u, n, inv, LV.r0);
    W.L = L0;
    W.Lc = 0.f;
    W.tau = tau0;
    if constexpr (TwoBin<Cell>::value) {
        W.Ln = (l == A.level0) ? __ldg(A.srcLn + s) : __ldcg(B.Ln + i);
        W.Lnc = 0.f;
        W.taun = (l == A.level0) ? 0.f : __ldcg(B.taun + i);
    }
    W.cell = inside ? load_cell(cells + W.idx) : cell_zero<Cell>();
    return inside ? 1 : 0;
}

// Marks the four child slots of parent slot c4/4 as empty.
__device__ __forceinline__ void write_holes(const RayBuf& C, unsigned long long c4)
{
    if (c4 + 4 <= C.cap)
        *reinterpret_cast<uint4*>(C.src + c4) = make_uint4(kHole, kHole, kHole, kHole);
}

// Adds a warp's count of rays started at level l to the per-level counters.
__device__ __forceinline__ void count_rays(DevStats* st, int l, unsigned n)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) n += __shfl_down_sync(kFull, n, off);
    if ((threadIdx.x & 31u) == 0 && n > 0) {
        atomicAdd(&st->rays_per_level[l], (unsigned long long)n);
        atomicAdd(&st->rays_total, (unsigned long long)n);
        atomicMax(&st->level_reached, l);
    }
}

// Grid-wide barrier for a cooperative launch. Every wait is bounded by wait_ns of
// %globaltimer; on expiry the block records ART_ETIMEOUT and the barrier returns false.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool grid_barrier(Sched* sc, DevStats* st, long long wait_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = &sc->bar_gen;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&sc->bar_count, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(&sc->bar_count, 0u);
            __threadfence();
            atomicAdd(&sc->bar_gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g) {
                if (wait_ns < 0 || (long long)(global_ns() - t0) > wait_ns) {
                    atomicCAS(&st->error, 0, -4);  // ART_ETIMEOUT
                    ok = 0;
                    break;
                }
                __nanosleep(200);
            }
        }
        __threadfence();
        if (*((volatile int*)&st->error) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace art
