// art_kernels.cuh -- forward trace kernels of the GB300 adaptive ray trace.
//
// Work decomposition. The rays of one HEALPix level form a "front" held structure-of-arrays
// in a level buffer. A warp takes rays from the front in chunks (one ray per lane, lanes
// refill from the chunk as their rays end), walks each ray from its start radius to its end
// (Sec. 2.1: r_max(l), tau > tau_max or the grid boundary) and appends the four children of
// every split ray to the next level's buffer with one warp-aggregated reservation.
//
// Two schedules share that routine:
//   * plain: one launch per (source, level), fronts kept whole;
//   * persistent: one cooperative launch for all sources. The launch loops over phases;
//     each phase consumes the top part of the deepest non-empty level buffer, at most a
//     quarter of the next buffer's capacity, so the children always fit. Deepest-first order
//     keeps every buffer bounded, which is the memory role the paper's last-in-first-out ray
//     stack plays (Sec. 2.2). A grid barrier with a bounded wait separates phases; the
//     retired-ray weights 4^(l_max - l) are summed as the paper's destroy counter (Sec. 2.2).
#pragma once

#include "art_device.cuh"

namespace art {

// ---------------------------------------------------------------------------------------
// HEALPix nested directions in FP64 (Gorski et al. 2005), rotated, split into hi + lo
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t even_bits(uint64_t x)
{
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x >> 4)) & 0x00ff00ff00ff00ffull;
    x = (x | (x >> 8)) & 0x0000ffff0000ffffull;
    x = (x | (x >> 16)) & 0x00000000ffffffffull;
    return (uint32_t)x;
}

// cos and sin of pi * num / den (den > 0), exact at multiples of 1/2, cos = sin at 1/4.
__device__ __forceinline__ void cossin_pi_frac(long long num, long long den, double& c, double& s)
{
    long long m = num % (2 * den);
    if (m < 0) m += 2 * den;
    double sgn_c = 1.0, sgn_s = 1.0;
    if (m >= den) { m -= den; sgn_c = -1.0; sgn_s = -1.0; }  // shift by pi
    if (2 * m > den) { m = den - m; sgn_c = -sgn_c; }        // reflect about pi/2
    double cv, sv;
    if (m == 0) { cv = 1.0; sv = 0.0; }
    else if (2 * m == den) { cv = 0.0; sv = 1.0; }
    else if (4 * m == den) { cv = 0.70710678118654752440; sv = cv; }
    else sincospi((double)m / (double)den, &sv, &cv);
    c = sgn_c * cv;
    s = sgn_s * sv;
}

__global__ void k_directions(int level, unsigned long long npix, double r0, double r1, double r2,
                             double r3, double r4, double r5, double r6, double r7, double r8,
                             int rotate, float4* __restrict__ dir)
{
    unsigned long long p = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const long long ns = 1ll << level;
    const unsigned long long nface = (unsigned long long)(ns * ns);
    const int face = (int)(p / nface);
    const unsigned long long q = p - (unsigned long long)face * nface;
    const long long x = even_bits(q), y = even_bits(q >> 1);
    const int row = face >> 2;                      // 0 north, 1 equator, 2 south
    const long long ring = (long long)(row + 2) * ns - x - y - 1;
    long long nr;
    int shift = 0;
    double z, st;
    if (ring < ns || ring > 3 * ns) {
        nr = ring < ns ? ring : 4 * ns - ring;
        double a = (double)(nr * nr) / (3.0 * (double)(ns * ns));
        z = ring < ns ? 1.0 - a : a - 1.0;
        st = sqrt(a * (2.0 - a));
    } else {
        nr = ns;
        shift = (int)((ring - ns) & 1);
        z = (double)(4 * ns - 2 * ring) / (3.0 * (double)ns);
        st = sqrt((1.0 - z) * (1.0 + z));
    }
    const int col = (row == 1) ? 2 * (face & 3) : 2 * (face & 3) + 1;
    long long jp = (col * nr + x - y + 1 + shift) / 2;
    if (jp > 4 * nr) jp -= 4 * nr;
    if (jp < 1) jp += 4 * nr;
    double c, s;
    cossin_pi_frac(2 * jp - shift - 1, 4 * nr, c, s);
    double v[3] = {st * c, st * s, z};
    double w[3];
    if (rotate) {
        w[0] = r0 * v[0] + r1 * v[1] + r2 * v[2];
        w[1] = r3 * v[0] + r4 * v[1] + r5 * v[2];
        w[2] = r6 * v[0] + r7 * v[1] + r8 * v[2];
    } else {
        w[0] = v[0]; w[1] = v[1]; w[2] = v[2];
    }
    float h[3], l[3], ih[3], il[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (fabs(w[a]) < 5.9604644775390625e-08) w[a] = 0.0;  // 2^-24
        h[a] = __double2float_rn(w[a]);
        l[a] = __double2float_rn(w[a] - (double)h[a]);
        const double iv = w[a] != 0.0 ? 1.0 / w[a] : 0.0;
        ih[a] = __double2float_rn(iv);
        il[a] = __double2float_rn(iv - (double)ih[a]);
    }
    // layout: {n_hx, n_hy, n_hz, n_lx}, {n_ly, n_lz, i_hx, i_hy}, {i_hz, i_lx, i_ly, i_lz}
    dir[3 * p] = make_float4(h[0], h[1], h[2], l[0]);
    dir[3 * p + 1] = make_float4(l[1], l[2], ih[0], ih[1]);
    dir[3 * p + 2] = make_float4(ih[2], il[0], il[1], il[2]);
}

// chi per cell length (dx) in FP32 from the density fields, in the padded layout with the
// sentinel ring; flags bad densities.
__global__ void k_opacity(int nx, int ny, int nz, const float* __restrict__ nH0,
                          const float* __restrict__ nH, double sH_dx, double sd_dx,
                          float* __restrict__ chi, float2* __restrict__ chi2,
                          DevStats* __restrict__ st)
{
    const unsigned npad = (unsigned)(nx + 2) * (unsigned)(ny + 2) * (unsigned)(nz + 2);
    const unsigned step = gridDim.x * blockDim.x;
    bool bad = false;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < npad; q += step) {
        unsigned i;
        if (!unpad(q, nx, ny, nz, i)) {
            chi[q] = kSentinel;
            if (chi2) chi2[q] = make_float2(kSentinel, 0.f);
            continue;
        }
        float a = nH0[i];
        float b = nH ? nH[i] : 0.f;
        bad = bad || !(a >= 0.f) || !(b >= 0.f) || isinf(a) || isinf(b);
        double h = (double)a * sH_dx;
        const double dust = (double)b * sd_dx;
        chi[q] = __double2float_rn(h + dust);
        if (chi2) chi2[q] = make_float2(__double2float_rn(h + dust), __double2float_rn(dust));
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicCAS(&st->error, 0, -1);
}

// Level-l0 rays of sources [s0, s0 + ns): pixel-major within each source.
__global__ void k_inject(int s0, int nsrc, unsigned npix0, RayBuf B, unsigned long long* count)
{
    unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    unsigned long long n = (unsigned long long)nsrc * npix0;
    if (i == 0) *count = n;
    if (i >= n) return;
    unsigned s = (unsigned)(i / npix0);
    unsigned p = (unsigned)(i - (unsigned long long)s * npix0);
    B.src[i] = s0 + s;
    B.pix[i] = p;
    B.L[i] = 0.f;     // filled from the source table when the ray starts
    B.tau[i] = 0.f;
}

// Processes the rays in slots [cursor .. end) of level l, whose phase starts at slot
// `begin` (cursor advanced atomically by warps, `chunk` slots at a time). The children of
// the ray in slot i go to slots 4 (i - begin) .. +3 of level l + 1, so the next front keeps
// the pixel order of this one; parents that do not split mark their four slots empty. Idle
// lanes are refilled once 16 of the 32 are idle, so the ray set-up runs with many lanes at
// once. Warp-uniform: every lane of the warp must call it.
// The per-cell records a trace gathers: opacities (one bin) or opacity pairs (two bins).
template <class Cell> __device__ __forceinline__ const Cell* cells_of(const TraceArgs& A);
template <> __device__ __forceinline__ const float* cells_of<float>(const TraceArgs& A) { return A.chi; }
template <> __device__ __forceinline__ const float2* cells_of<float2>(const TraceArgs& A) { return A.chi2; }

// Idle lanes of a warp before it refills them from its chunk, and steps between refill
// checks (measured: 16 lanes > 18, 14 > 12 > 10; 64 steps > 32 > 16 > 8).
#ifndef ART_FWD_IDLE
#define ART_FWD_IDLE 16
#endif
#ifndef ART_FWD_STEPS
#define ART_FWD_STEPS 64
#endif

template <class Cell, bool kCut>
__device__ void run_rays(const TraceArgs& A, const Cell* cells, int l,
                         unsigned long long* cursor, unsigned long long begin,
                         unsigned long long end, Tally& T)
{
    constexpr bool two = TwoBin<Cell>::value;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = (1u << lane) - 1u;
    const LevelInfo& LV = A.levels[l];
    const df lv_rmax = LV.rmax;  // split radius of this level, kept in registers
    const RayBuf& B = A.buf[l];
    const RayBuf& C = A.buf[l + 1];
    const bool has_next = l < A.lmax_glob;

    // slot indices fit in 32 bits (level buffers hold fewer than 2^31 slots)
    const unsigned b32 = (unsigned)begin, e32 = (unsigned)end;
    unsigned wnext = 0, wend = 0;
    bool more = true;
    bool active = false;
    WalkT<Cell> W;
    unsigned s = 0, p = 0;
    unsigned slot = 0;
    float L0 = 0.f;
    bool splits = false;
    bool first = false;  // next step is the first segment of a base-level ray
    const bool base = l == A.level0;
    unsigned ncross = 0, nrays = 0;

    for (;;) {
        // refill idle lanes from the warp's chunk, fetching chunks as needed
        unsigned need = __ballot_sync(kFull, !active);
        if (__popc(need) >= ART_FWD_IDLE || need == kFull) {
            while (need && more) {
                if (wnext >= wend) {
                    unsigned long long b = 0;
                    if (lane == 0) b = atomicAdd(cursor, (unsigned long long)A.chunk);
                    b = __shfl_sync(kFull, b, 0);
                    if (b >= end) { more = false; break; }
                    wnext = (unsigned)b;
                    wend = min(wnext + (unsigned)A.chunk, e32);
                }
                const unsigned avail = min(wend - wnext, 32u);
                const unsigned rank = __popc(need & lt);
                if (!active && rank < avail) {
                    slot = wnext + rank;
                    const int st = ray_begin(A, LV, B, l, slot, W, cells, s, p, L0, splits);
                    if (st > 0) {
                        active = true;
                        first = base;
                        ++nrays;
                    } else {
                        if (st == 0) {  // starts outside the grid: escapes with its full L
                            atomicAdd(&T.escaped, (double)L0);
                            if constexpr (two) atomicAdd(&T.escaped_n, (double)W.Ln + (double)W.Lnc);
                            atomicAdd(&T.destroy, LV.destroy_w);
                            ++nrays;
                        }
                        if (has_next) write_holes(C, 4ull * (slot - b32));
                    }
                }
                wnext += min(avail, (unsigned)__popc(need));
                need = __ballot_sync(kFull, !active);
            }
        }
        if (!__any_sync(kFull, active)) {
            if (!more) break;
            continue;
        }

#pragma unroll 1
        for (int k = 0; k < ART_FWD_STEPS; ++k) {
            bool dep = false;
            int cell = 0;
            float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (active) {
                // a ray ends at a radius when it can split or (kCut) at the d_max cutoff
                StepOut o;
                if constexpr (kCut)
                    o = walk_step<false>(W, true, end_radius(splits, lv_rmax, A.dmax), cells,
                                         A.tau_max);
                else
                    o = walk_step<false>(W, splits, lv_rmax, cells, A.tau_max);
                dep = o.seg;  // segments without length deposit nothing
                cell = o.cell;
                const float dm = two ? o.dL + o.dLn : o.dL;  // momentum of both bins
                dv = make_float4(o.G, dm * W.n[0], dm * W.n[1], dm * W.n[2]);
                ncross += o.seg ? 1u : 0u;
                if (o.end) {
                    active = false;
                    const unsigned long long c4 = 4ull * (slot - b32);
                    if (o.ev == EV_SPLIT && (!kCut || splits_at_end(splits, LV.rmax, A.dmax))) {
                        if (c4 + 4 <= C.cap) {
                            const float Lc = 0.25f * W.L;
                            *reinterpret_cast<uint4*>(C.src + c4) = make_uint4(s, s, s, s);
                            *reinterpret_cast<uint4*>(C.pix + c4) =
                                make_uint4(4 * p, 4 * p + 1, 4 * p + 2, 4 * p + 3);
                            *reinterpret_cast<float4*>(C.L + c4) = make_float4(Lc, Lc, Lc, Lc);
                            *reinterpret_cast<float4*>(C.tau + c4) =
                                make_float4(W.tau, W.tau, W.tau, W.tau);
                            if constexpr (two) {
                                const float Ln = 0.25f * W.Ln;
                                *reinterpret_cast<float4*>(C.Ln + c4) = make_float4(Ln, Ln, Ln, Ln);
                                *reinterpret_cast<float4*>(C.taun + c4) =
                                    make_float4(W.taun, W.taun, W.taun, W.taun);
                            }
                        } else {
                            atomicCAS(&A.stats->error, 0, -3);  // ART_EQUEUE_OVERFLOW
                        }
                        // the split ray's ledger residual: its children start from L itself
                        if (W.Lc != 0.f) atomicAdd(&T.escaped, (double)W.Lc);
                        if constexpr (two) {
                            if (W.Lnc != 0.f) atomicAdd(&T.escaped_n, (double)W.Lnc);
                        }
                    } else {
                        // leaving the box or cut at d_max: escaped; tau > tau_max: dropped
                        const double Lend = (double)W.L + (double)W.Lc;
                        if (o.ev != EV_DROP) atomicAdd(&T.escaped, Lend);
                        else atomicAdd(&T.dropped, Lend);
                        if constexpr (two) {
                            const double Lnend = (double)W.Ln + (double)W.Lnc;
                            if (o.ev != EV_DROP) atomicAdd(&T.escaped_n, Lnend);
                            else atomicAdd(&T.dropped_n, Lnend);
                        }
                        atomicAdd(&T.destroy, LV.destroy_w);
                        if (has_next) write_holes(C, c4);
                    }
                }
            }
            if (base && __any_sync(kFull, first)) deposit_merged(A.acc, dep ? cell : -1, dv);
            else deposit_if(A.acc, dep, cell, dv);
            first = false;
        }
    }
    tally_crossings(T, ncross);
    count_rays(A.stats, l, nrays);
}

// Plain schedule: all slots of level l (one source's front).
// Launch bounds of the trace kernels: at most ART_TRACE_MAX_THREADS threads per block and
// ART_TRACE_MIN_BLOCKS resident blocks per SM, which caps the registers per thread at
// 65536 / (threads x blocks).
#ifndef ART_TRACE_MAX_THREADS
#define ART_TRACE_MAX_THREADS 512
#endif
#ifndef ART_TRACE_MIN_BLOCKS
#define ART_TRACE_MIN_BLOCKS 2
#endif
constexpr int kTraceMaxThreads = ART_TRACE_MAX_THREADS;

template <class Cell, bool kCut>
__global__ void __launch_bounds__(ART_TRACE_MAX_THREADS, ART_TRACE_MIN_BLOCKS) k_trace_level(const __grid_constant__ TraceArgs A, int l)
{
    tally_init();
    Tally& T = tally_slots()[threadIdx.x >> 5];
    // a front that overflowed (status set by the writer) is cut at the buffer capacity
    const unsigned long long end =
        min(*((volatile unsigned long long*)&A.sched->count[l]), A.buf[l].cap);
    if (blockIdx.x == 0 && threadIdx.x == 0 && l < A.lmax_glob) A.sched->count[l + 1] = 4 * end;
    run_rays<Cell, kCut>(A, cells_of<Cell>(A), l, &A.sched->cursor[l], 0, end, T);
    tally_flush(A.stats);
}

// Resets the per-level counters of the plain schedule before the next source.
__global__ void k_reset_counts(Sched* sc)
{
    int t = threadIdx.x;
    if (t < kNL) { sc->count[t] = 0; sc->cursor[t] = 0; }
}

// Persistent schedule: all sources, all levels, one cooperative launch.
template <class Cell, bool kCut>
__global__ void __launch_bounds__(ART_TRACE_MAX_THREADS, ART_TRACE_MIN_BLOCKS) k_trace_persistent(const __grid_constant__ TraceArgs A)
{
    tally_init();
    Tally& T = tally_slots()[threadIdx.x >> 5];
    Sched* sc = A.sched;
    __shared__ int s_level;
    __shared__ unsigned long long s_begin, s_end;
    for (;;) {
        if (!grid_barrier(sc, A.stats, A.wait_ns)) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            volatile unsigned long long* cnt = sc->count;
            int l = -1;
            for (int k = A.lmax_glob; k >= A.level0; --k)
                if (cnt[k] > 0) { l = k; break; }
            if (l < 0) {
                sc->done = 1;
            } else {
                unsigned long long have = min(cnt[l], A.buf[l].cap);
                unsigned long long take = have;
                if (l < A.lmax_glob) take = min(have, A.buf[l + 1].cap / 4);
                if (take == 0) {  // a phase must consume rays, or the schedule never ends
                    atomicCAS(&A.stats->error, 0, -8);  // ART_EINTERNAL
                    take = have;
                }
                sc->phase_level = l;
                sc->phase_begin = have - take;
                sc->phase_end = have;
                sc->cursor[l] = have - take;
                cnt[l] = have - take;
                if (l < A.lmax_glob) cnt[l + 1] = 4 * take;  // the children's slots
            }
            __threadfence();
        }
        if (!grid_barrier(sc, A.stats, A.wait_ns)) break;
        if (threadIdx.x == 0) {
            volatile Sched* v = sc;
            s_level = v->done ? -1 : v->phase_level;
            s_begin = v->phase_begin;
            s_end = v->phase_end;
        }
        __syncthreads();
        const int l = s_level;
        if (l < 0) break;
        run_rays<Cell, kCut>(A, cells_of<Cell>(A), l, &sc->cursor[l], s_begin, s_end, T);
    }
    tally_flush(A.stats);
}

// Gamma, force and energy from the accumulator (padded layout) into the caller's SoA
// outputs (nx*ny*nz layout).
__global__ void k_finalize(int nx, int ny, int nz, const float4* __restrict__ acc, float gscale,
                           float fscale, float escale, float* __restrict__ gamma,
                           float* __restrict__ force, float* __restrict__ energy)
{
    const unsigned ncell = (unsigned)nx * (unsigned)ny * (unsigned)nz;
    const unsigned step = gridDim.x * blockDim.x;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += step) {
        const float4 a = __ldcs(acc + pad_of(i, nx, ny));
        gamma[i] = gscale * a.x;
        if (force) {
            force[i] = fscale * a.y;
            force[(size_t)ncell + i] = fscale * a.z;
            force[2 * (size_t)ncell + i] = fscale * a.w;
        }
        if (energy) energy[i] = escale * a.x;
    }
}

}  // namespace art
