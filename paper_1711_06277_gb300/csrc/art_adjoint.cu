// art_adjoint.cu -- hand-written adjoint of the forward trace for
// loss = sum_c (w_c gamma_c + v_c . force_c) (new; the paper has no adjoint). Gradients with
// respect to log n_H0 per cell and to every source luminosity.
//
// For a segment j of a ray in cell c, with G_j = L_in ds phi(dtau), dL_j = L_in (1 - e^-dtau),
// dtau = chi ds and dtauH = n_H0 sigma_H ds (the part of dtau that scales with n_H0), the
// segment adds w_c k G_j + q_j dL_j to the loss (k converts G to gamma, q_j = (v_c . n)/dV)
// and
//   d loss / d log n_H0[c] += dtauH (w_c k L_in ds phi'(dtau) + q_j L_in e^-dtau - S_after(j)),
// where S_after(j) is the loss of every later segment of the ray and of all of its
// descendants (their entering luminosity carries the factor e^-dtau of segment j). Split
// points and tau_max retirement are held fixed.
//
// Nothing is stored per segment. Rays are traced with unit source luminosity (the loss is
// linear in each L_s; gradients are scaled by L_s when deposited) in the deepest-first phases
// of the persistent schedule, and every ray is walked twice:
//   pass 1 sums the ray's own weighted G; a ray that splits stores that sum, a count of 4
//     pending children and its children (with a back-pointer to it);
//   pass 2 (S = own sum + the children's totals) deposits the gradients and adds the ray's
//     total to its parent's. A ray that ends without splitting runs pass 2 at once; the lane
//     whose child brings a parent's pending count to zero runs the parent's pass 2, and so on
//     towards the base level.
// Children always finish before their parent's pass 2 because the count only reaches zero
// after all four of them have added their totals.
#include <cmath>
#include <algorithm>
#include <cstring>

#include "art.h"
#include "art_internal.h"

using namespace art;

namespace {


// Running sum in two floats without renormalisation: hi + g is split exactly (two-sum) and
// its rounding error collected in lo.
__device__ __forceinline__ df df_acc(df a, float g)
{
    const df s = df_two_sum(a.hi, g);
    return {s.hi, a.lo + s.lo};
}

// a - g for a remainder that only decreases (a >= g >= 0): with |hi| >= g the error of
// hi - g is exact by the fast two-sum; where rounding of earlier steps left hi just below g,
// hi - g is itself exact (Sterbenz) and the error is 0.
__device__ __forceinline__ df df_dec(df a, float g)
{
    const float s = a.hi - g;
    const float e = (a.hi - s) - g;
    return {s, a.lo + e};
}

// Per-lane sum of dloss/dL for the source of the lane's recent rays, flushed to the global
// FP64 sum when the lane moves to another source (rays of one source are consecutive).
struct DLacc {
    df v;
    unsigned src;
};

__device__ __forceinline__ void dl_add(DLacc& D, double* dL, unsigned s, df own)
{
    if (s != D.src) {
        if (D.src != 0xffffffffu && D.v.hi != 0.f) atomicAdd(dL + D.src, (double)D.v.hi + (double)D.v.lo);
        D.src = s;
        D.v = {0.f, 0.f};
    }
    D.v = df_add(D.v, own);
}

__device__ __forceinline__ void red_f32(float* p, float v)
{
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

// The {chi, chi_H, w, 0} part of a reverse-sweep cell record, and the force weight of the
// segment: q = (v . n) / dV, so that the segment adds q dL to the loss (0 without a force term).
__device__ __forceinline__ float4 rec_main(const float4& c) { return c; }
__device__ __forceinline__ float4 rec_main(const CellF& c) { return c.a; }
__device__ __forceinline__ float4 rec_main(const CellW& c) { return make_float4(c.chi, c.chi, c.w, 0.f); }
__device__ __forceinline__ float force_weight(const float4&, const float*, float) { return 0.f; }
__device__ __forceinline__ float force_weight(const CellW&, const float*, float) { return 0.f; }
__device__ __forceinline__ float force_weight(const CellF& c, const float* n, float fs)
{
    return fs * fmaf(c.b.x, n[0], fmaf(c.b.y, n[1], c.b.z * n[2]));
}
template <class Cell> __device__ __forceinline__ const Cell* recs_of(const TraceArgs& A);
template <> __device__ __forceinline__ const float4* recs_of<float4>(const TraceArgs& A) { return A.rec; }
template <> __device__ __forceinline__ const CellF* recs_of<CellF>(const TraceArgs& A) { return A.recf; }
template <> __device__ __forceinline__ const CellW* recs_of<CellW>(const TraceArgs& A) { return A.recw; }

// Idle lanes of a warp before it refills them from the queue, and steps per round (between
// refill checks; completions run at the end of each round). Measured on the 128^3 /
// 16-source and 512^3 / 8-source cases: 32 steps at 16 lanes beat 8 at 12 by 1 % and 10 %;
// longer rounds or a threshold of 20 lanes gain a little more at 512^3 and lose at 128^3.
#ifndef ART_ADJ_IDLE
#define ART_ADJ_IDLE 16
#endif
#ifndef ART_ADJ_STEPS
#define ART_ADJ_STEPS 32
#endif

// One expand phase of the reverse sweep on the rays in slots [cursor .. end) of level l
// (phase starting at slot `begin`). Pass 1 walks each ray for its own weighted sum. A ray
// that splits stores that sum, a pending-children count of 4 and its children (in order, as
// in the forward trace). A ray that ends without splitting (a leaf) walks again at once
// (pass 2) from the start state kept from pass 1, depositing its gradients; once the warp's
// round of steps ends it adds its total to its parent and counts the parent down (the
// completions of a round run together). The lane that brings a parent's
// count to zero takes over the parent's pass 2 (its level below this phase's), and so on
// towards the base level: no separate collapse phase is needed, because the deepest-first
// schedule does not reuse a level's slots before everything below it has finished. The
// level data and buffer descriptors are copied out of the kernel parameters here: a
// rewrite of the completion step that held references into the parameter block, indexed
// by the changing level lv, never finished on the GPU with the d_max cutoff (the same
// inputs finish in 2 ms with this form). Warp-uniform.
template <class Cell, bool kCut>
__device__ void run_adjoint(const TraceArgs& A, int l, unsigned long long* cursor,
                            unsigned long long begin, unsigned long long end, Tally& T, DLacc& D)
{
    const Cell* const recs = recs_of<Cell>(A);
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = (1u << lane) - 1u;
    const LevelInfo LV = A.levels[l];
    const RayBuf B = A.buf[l];
    const RayBuf C = A.buf[l + 1];
    const bool has_next = l < A.lmax_glob;
    const float gs = A.gscale;

    // slot indices fit in 32 bits (level buffers hold fewer than 2^31 slots)
    const unsigned b32 = (unsigned)begin, e32 = (unsigned)end;
    unsigned wnext = 0, wend = 0;
    bool more = true;
    int mode = 0;          // 0 idle, 1 pass 1 (level l), 2 pass 2 (level lv <= l),
                           // 3 pass 2 ended, completion pending
    int lv = l;            // level of the ray being walked
    WalkT<Cell> W;
    // pass-1 start of the ray (next face per axis, start cell), so that a leaf's pass 2
    // restarts without a new ray set-up
    df t0[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    int idx0 = 0;
    unsigned s = 0, p = 0;
    unsigned slot = 0;
    float L0 = 0.f, Ls = 0.f;
    df own = {0.f, 0.f};   // own weighted sum (pass 1), kept for dL in pass 2
    float total = 0.f;     // own + descendants (pass 2), passed to the parent
    df rem = {0.f, 0.f};   // weighted sum over what follows the current segment (pass 2)
    df rmax = LV.rmax;     // radius where the ray of level lv ends (split or cutoff)
    bool splits = false;
    unsigned ncross = 0, nrays = 0;
    // Every step crosses at least one face and the sentinel ring ends every walk that
    // leaves the grid, so walks end by construction. As a safety net the warp counts its
    // rounds of steps (ART_ADJ_STEPS each) and gives up past a bound far beyond any phase
    // (ART_EINTERNAL), so the kernel always ends.
    unsigned rounds = 0;
    unsigned nretired = 0;  // rays retired here (weight destroy_w each, summed at the end)

    // Completion of the ray in `slot` at level lv (pass 2 done, or a ray without segments):
    // dL, the parent's sum, and possibly the parent's pass 2 in this lane.
    auto complete = [&]() {
        for (;;) {
            dl_add(D, A.dL, s, own);  // every ray of the chain has source s
            if (lv == A.level0) { mode = 0; return; }
            const RayBuf Bl = A.buf[lv];
            const RayBuf Pl = A.buf[lv - 1];
            const unsigned par = __ldcg(Bl.parent + slot);
            if (total != 0.f) red_f32(Pl.sub + par, total);
            // count the parent down with acquire-release ordering: this ray's sum (above) is
            // released with the decrement, and the lane that takes the count to zero acquires
            // every sibling's sum before reading the parent's total
            unsigned old;
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                         : "=r"(old) : "l"(Pl.pending + par), "r"(0xffffffffu) : "memory");
            if (old != 1u) { mode = 0; return; }
            // last child: this lane replays the parent (pass 2)
            lv -= 1;
            slot = par;
            const float2 ov = __ldcg(Pl.own + slot);
            own = {ov.x, ov.y};
            rem = df_add(own, {__ldcg(Pl.sub + slot), 0.f});
            total = rem.hi + rem.lo;
            const LevelInfo Lp = A.levels[lv];
            if constexpr (!kCut) rmax = Lp.rmax;
            ray_begin(A, Lp, Pl, lv, slot, W, recs, s, p, L0, splits);
            if constexpr (kCut) rmax = end_radius(splits, Lp.rmax, A.dmax);
            Ls = __ldg(A.srcL + s);
            mode = 2;
            return;
        }
    };

    for (;;) {
        unsigned need = __ballot_sync(kFull, mode == 0);
        if (__popc(need) >= ART_ADJ_IDLE || need == kFull) {
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
                if (mode == 0 && rank < avail) {
                    slot = wnext + rank;
                    lv = l;
                    if constexpr (!kCut) rmax = LV.rmax;
                    const int st = ray_begin(A, LV, B, l, slot, W, recs, s, p, L0, splits);
                    if constexpr (kCut) rmax = end_radius(splits, LV.rmax, A.dmax);
                    if (st > 0) {
                        Ls = __ldg(A.srcL + s);
                        t0[0] = W.t[0];
                        t0[1] = W.t[1];
                        t0[2] = W.t[2];
                        idx0 = W.idx;
                        mode = 1;
                        own = {0.f, 0.f};
                        ++nrays;
                    } else {
                        if (has_next) write_holes(C, 4ull * (slot - b32));
                        if (st == 0) {  // starts outside the grid: a leaf with zero sums
                            ++nretired;
                            ++nrays;
                            own = {0.f, 0.f};
                            total = 0.f;
                            complete();
                        }
                    }
                }
                wnext += min(avail, (unsigned)__popc(need));
                need = __ballot_sync(kFull, mode == 0);
            }
        }
        if (!__any_sync(kFull, mode != 0)) {
            if (!more) break;
            continue;
        }

        if (++rounds > (1u << 28)) {  // warp-uniform: no phase comes near this
            if (lane == 0) atomicCAS(&A.stats->error, 0, -8);  // ART_EINTERNAL
            break;
        }
#pragma unroll 1
        for (int k = 0; k < ART_ADJ_STEPS; ++k) {
            if (mode == 1 || mode == 2) {
                const float4 cm = rec_main(W.cell);
                const float wv = cm.z;   // weight and neutral-H opacity of this cell
                const float hv = cm.y;
                const float q = force_weight(W.cell, W.n, A.fscale);
                // a ray ends at a radius (rmax) when it can split or (kCut) at the cutoff
                const StepOut o = walk_step<false, true>(W, kCut || splits, rmax, recs, A.tau_max);
                // this segment's loss: w k G, plus q dL with a force term
                const float g = fmaf(q, o.dL, wv * gs * o.G);
                if (mode == 1) {
                    own = df_acc(own, g);
                    ncross += o.seg ? 1u : 0u;
                } else {
                    rem = df_dec(rem, g);
                    const float after = rem.hi + rem.lo;
                    // d(segment loss)/d dtau: w k L_in ds phi' + q L_in e^-dtau (W.L is now
                    // L_in e^-dtau)
                    const float own_d = fmaf(q, W.L, wv * gs * o.Lin * o.ds * o.dphi);
                    const float val = Ls * hv * o.ds * (own_d - after);
                    if (o.seg) red_f32(A.grad + o.cell, val);
                }
                if (o.ev != EV_NONE) {
                    if (mode == 1) {
                        const unsigned long long c4 = 4ull * (slot - b32);
                        if (o.ev == EV_SPLIT && (!kCut || splits_at_end(splits, LV.rmax, A.dmax))) {
                            B.own[slot] = make_float2(own.hi, own.lo);
                            B.sub[slot] = 0.f;
                            B.pending[slot] = 4u;
                            if (c4 + 4 <= C.cap) {
                                const float Lc = 0.25f * W.L;
                                *reinterpret_cast<uint4*>(C.src + c4) = make_uint4(s, s, s, s);
                                *reinterpret_cast<uint4*>(C.pix + c4) =
                                    make_uint4(4 * p, 4 * p + 1, 4 * p + 2, 4 * p + 3);
                                *reinterpret_cast<float4*>(C.L + c4) = make_float4(Lc, Lc, Lc, Lc);
                                *reinterpret_cast<float4*>(C.tau + c4) =
                                    make_float4(W.tau, W.tau, W.tau, W.tau);
                                *reinterpret_cast<uint4*>(C.parent + c4) =
                                    make_uint4(slot, slot, slot, slot);
                            } else {
                                atomicCAS(&A.stats->error, 0, -3);
                            }
                            mode = 0;
                        } else {
                            ++nretired;
                            if (has_next) write_holes(C, c4);
                            // a leaf: pass 2 right away
                            total = own.hi + own.lo;
                            rem = own;
                            // a leaf: pass 2 right away, from the kept start state (direction
                            // steps, source and luminosity are the ray's own already)
                            W.t[0] = t0[0];
                            W.t[1] = t0[1];
                            W.t[2] = t0[2];
                            W.idx = idx0;
                            W.tc = LV.r0;
                            W.L = L0;
                            W.Lc = 0.f;
                            W.tau = l == A.level0 ? 0.f : __ldcg(B.tau + slot);
                            W.cell = load_cell(recs + idx0);
                            mode = 2;
                        }
                    } else {
                        mode = 3;
                    }
                }
            }
        }
        // Completions of the round's finished pass-2 walks run together: the count-down of
        // the parent with its memory ordering, and the set-up of the parent's pass 2 for a
        // last child, whose latencies then overlap across lanes (measured 4 % faster than
        // completing each walk in its own step, and faster than batches of 1 to 8 lanes, in
        // rounds of 8 steps).
        if (mode == 3) complete();
    }
    tally_crossings(T, ncross);
    count_rays(A.stats, l, nrays);
    // the destroy counter: rays retired at this phase's level, weight 4^(l_max - l)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nretired += __shfl_down_sync(kFull, nretired, off);
    if (lane == 0 && nretired > 0) atomicAdd(&T.destroy, (unsigned long long)nretired * LV.destroy_w);
}

template <class Cell, bool kCut>
__global__ void __launch_bounds__(256, 4) k_backward_persistent(const __grid_constant__ TraceArgs A)
{
    tally_init();
    Tally& T = tally_slots()[threadIdx.x >> 5];
    DLacc D = {{0.f, 0.f}, 0xffffffffu};
    Sched* sc = A.sched;
    __shared__ int s_level;
    __shared__ unsigned long long s_begin, s_end;
    for (;;) {
        if (!grid_barrier(sc, A.stats, A.wait_ns)) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            volatile Sched* v = sc;
            int l = -1;
            for (int k = A.lmax_glob; k >= A.level0; --k)
                if (v->count[k] > 0) { l = k; break; }
            if (l < 0) {
                v->done = 1;
            } else {
                const unsigned long long have = min(v->count[l], A.buf[l].cap);
                unsigned long long take = have;
                if (l < A.lmax_glob) take = min(have, A.buf[l + 1].cap / 4);
                if (take == 0) {  // a phase must consume rays, or the schedule never ends
                    atomicCAS(&A.stats->error, 0, -8);  // ART_EINTERNAL
                    take = have;
                }
                const unsigned long long b = have - take;
                v->count[l] = b;
                v->phase_level = l;
                v->phase_begin = b;
                v->phase_end = have;
                v->cursor[l] = b;
                if (l < A.lmax_glob) v->count[l + 1] = 4 * take;  // the children's slots
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
        run_adjoint<Cell, kCut>(A, l, &sc->cursor[l], s_begin, s_end, T, D);
    }
    if (D.src != 0xffffffffu && D.v.hi != 0.f) atomicAdd(A.dL + D.src, (double)D.v.hi + (double)D.v.lo);
    tally_flush(A.stats);
}

// Per-cell record of the reverse sweep in the padded layout: one 16-byte gather per
// crossing, {chi, chi_H, w, 0} with chi and its neutral-H part formed exactly as k_opacity
// forms the forward trace's opacity; the sentinel ring holds {-1, 0, 0, 0}.
__global__ void k_pack_cells(int nx, int ny, int nz, const float* __restrict__ nH0,
                             const float* __restrict__ nH, double sH_dx, double sd_dx,
                             const float* __restrict__ w, float4* __restrict__ rec)
{
    const unsigned npad = (unsigned)(nx + 2) * (unsigned)(ny + 2) * (unsigned)(nz + 2);
    const unsigned step = gridDim.x * blockDim.x;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < npad; q += step) {
        unsigned i;
        if (!unpad(q, nx, ny, nz, i)) {
            rec[q] = make_float4(kSentinel, 0.f, 0.f, 0.f);
            continue;
        }
        const double h = (double)nH0[i] * sH_dx;
        const double dust = nH ? (double)nH[i] * sd_dx : 0.0;
        rec[q] = make_float4(__double2float_rn(h + dust), __double2float_rn(h), w ? w[i] : 0.f, 0.f);
    }
}

// The same with the force weight v (3 blocks of nx*ny*nz floats: x, y, z).
__global__ void k_pack_cells_f(int nx, int ny, int nz, const float* __restrict__ nH0,
                               const float* __restrict__ nH, double sH_dx, double sd_dx,
                               const float* __restrict__ w, const float* __restrict__ v,
                               CellF* __restrict__ rec)
{
    const unsigned npad = (unsigned)(nx + 2) * (unsigned)(ny + 2) * (unsigned)(nz + 2);
    const size_t ncell = (size_t)nx * ny * nz;
    const unsigned step = gridDim.x * blockDim.x;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < npad; q += step) {
        unsigned i;
        if (!unpad(q, nx, ny, nz, i)) {
            rec[q].a = make_float4(kSentinel, 0.f, 0.f, 0.f);
            rec[q].b = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const double h = (double)nH0[i] * sH_dx;
        const double dust = nH ? (double)nH[i] * sd_dx : 0.0;
        rec[q].a = make_float4(__double2float_rn(h + dust), __double2float_rn(h), w ? w[i] : 0.f, 0.f);
        rec[q].b = make_float4(v[i], v[ncell + i], v[2 * ncell + i], 0.f);
    }
}

// The 8-byte record {chi, w} of a sweep without dust and force term (sentinel {-1, 0}).
__global__ void k_pack_cells_w(int nx, int ny, int nz, const float* __restrict__ nH0,
                               double sH_dx, const float* __restrict__ w,
                               CellW* __restrict__ rec)
{
    const unsigned npad = (unsigned)(nx + 2) * (unsigned)(ny + 2) * (unsigned)(nz + 2);
    const unsigned step = gridDim.x * blockDim.x;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < npad; q += step) {
        unsigned i;
        if (!unpad(q, nx, ny, nz, i)) {
            rec[q] = CellW{kSentinel, 0.f};
            continue;
        }
        rec[q] = CellW{__double2float_rn((double)nH0[i] * sH_dx), w ? w[i] : 0.f};
    }
}

// Gradient per cell from the padded scratch it was summed in, into the caller's layout.
__global__ void k_unpad_grad(int nx, int ny, int nz, const float* __restrict__ src,
                             float* __restrict__ dst)
{
    const unsigned ncell = (unsigned)nx * (unsigned)ny * (unsigned)nz;
    const unsigned step = gridDim.x * blockDim.x;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += step)
        dst[i] = src[pad_of(i, nx, ny)];
}

__global__ void k_inject_all(int nsrc, unsigned npix0, RayBuf B, unsigned long long* count)
{
    unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    unsigned long long n = (unsigned long long)nsrc * npix0;
    if (i == 0) *count = n;
    if (i >= n) return;
    unsigned s = (unsigned)(i / npix0);
    B.src[i] = s;
    B.pix[i] = (unsigned)(i - (unsigned long long)s * npix0);
    B.L[i] = 0.f;
    B.tau[i] = 0.f;
}

int status_of(cudaError_t e)
{
    if (e == cudaSuccess) return ART_OK;
    return e == cudaErrorMemoryAllocation ? ART_ENOMEM : ART_ECUDA;
}

}  // namespace

extern "C" int art_trace_backward(art_grid* g, const art_params* p, const float* d_w,
                                  const float* d_v, float* d_dlog_nH0, double* d_dL,
                                  art_stats* h_stats)
{
    if (!g || (!d_w && !d_v) || !d_dlog_nH0) return ART_EINVAL;
    int rc = check_params(p);
    if (rc) return rc;
    // the reverse sweep always runs the persistent schedule (all base rays in one buffer)
    art_params pp = *p;
    pp.schedule = ART_SCHED_PERSISTENT;
    p = &pp;
    const int ns = (int)g->L.size();
    if (ns == 0) return ART_ESTATE;
    if (g->two_bin) return ART_EINVAL;  // the reverse sweep covers one-bin traces
    cudaStream_t st = g->stream;
    if ((rc = status_of(cudaMemsetAsync(g->d_stats, 0, sizeof(DevStats), st)))) return rc;
    rc = prepare_trace(g, p, true);
    if (rc) return rc;
    if ((size_t)ns > g->srcL_cap) {
        if (g->d_srcL) cudaFree(g->d_srcL);
        if (g->d_dL_scratch) cudaFree(g->d_dL_scratch);
        g->d_srcL = nullptr;
        g->d_dL_scratch = nullptr;
        g->srcL_cap = 0;
        if ((rc = status_of(cudaMalloc((void**)&g->d_srcL, sizeof(float) * ns)))) return rc;
        if ((rc = status_of(cudaMalloc((void**)&g->d_dL_scratch, sizeof(double) * ns)))) return rc;
        g->srcL_cap = ns;
    }
    g->h_srcL.resize(ns);
    for (int s = 0; s < ns; ++s) g->h_srcL[s] = (float)g->L[s];
    if ((rc = status_of(cudaMemcpyAsync(g->d_srcL, g->h_srcL.data(), sizeof(float) * ns,
                                        cudaMemcpyHostToDevice, st))))
        return rc;
    double* dL = d_dL ? d_dL : g->d_dL_scratch;
    if ((rc = status_of(cudaMemsetAsync(dL, 0, sizeof(double) * ns, st)))) return rc;
    // the gradient is summed in the padded layout, in the (otherwise idle) accumulator
    float* grad_pad = reinterpret_cast<float*>(g->d_acc);
    if ((rc = status_of(cudaMemsetAsync(grad_pad, 0, sizeof(float) * g->npad, st)))) return rc;
    if ((rc = status_of(cudaMemsetAsync(g->d_sched, 0, sizeof(Sched), st)))) return rc;
    const int l0 = p->level0;
    const unsigned npix0 = 12u << (2 * l0);
    const unsigned long long nb = (unsigned long long)ns * npix0;
    k_inject_all<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(ns, npix0, g->buf[l0],
                                                            &g->d_sched->count[l0]);
    if ((rc = status_of(cudaGetLastError()))) return rc;
    const int pack_blocks = (int)std::min<long long>((g->npad + 255) / 256, (long long)g->sms * 16);
    const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const double sH_dx = p->sigma_H * g->dx;
    const double sd_dx = g->nH ? p->sigma_d * g->dx : 0.0;
    // without dust the neutral-H opacity is the opacity: an 8-byte record serves
    const bool light = !d_v && sd_dx == 0.0;
    if (light) {
        if (!g->d_recw && (rc = status_of(cudaMalloc((void**)&g->d_recw, sizeof(CellW) * g->npad))))
            return rc;
        k_pack_cells_w<<<pack_blocks, 256, 0, st>>>(nx, ny, nz, g->nH0, sH_dx, d_w, g->d_recw);
    } else if (d_v) {
        if (!g->d_recf && (rc = status_of(cudaMalloc((void**)&g->d_recf, sizeof(CellF) * g->npad))))
            return rc;
        k_pack_cells_f<<<pack_blocks, 256, 0, st>>>(nx, ny, nz, g->nH0, g->nH, sH_dx, sd_dx, d_w,
                                                    d_v, g->d_recf);
    } else {
        if (!g->d_rec && (rc = status_of(cudaMalloc((void**)&g->d_rec, sizeof(float4) * g->npad))))
            return rc;
        k_pack_cells<<<pack_blocks, 256, 0, st>>>(nx, ny, nz, g->nH0, g->nH, sH_dx, sd_dx, d_w,
                                                  g->d_rec);
    }
    if ((rc = status_of(cudaGetLastError()))) return rc;
    TraceArgs A = make_args(g, p);
    A.rec = g->d_rec;
    A.recf = d_v ? g->d_recf : nullptr;
    A.recw = light ? g->d_recw : nullptr;
    A.w = d_w;
    A.grad = grad_pad;
    A.dL = dL;
    A.srcL = g->d_srcL;
    const double dV = g->dx * g->dx * g->dx;
    A.gscale = (float)(p->sigma_H * g->dx / dV);
    A.fscale = (float)(1.0 / dV);
    // the reverse sweep is compiled for blocks of at most 256 threads (register budget)
    const int threads = p->block_threads > 0 && p->block_threads < 256 ? p->block_threads : 256;
    const bool cut = p->d_max > 0.0;
    void (*kern)(TraceArgs) =
        light ? (cut ? k_backward_persistent<CellW, true> : k_backward_persistent<CellW, false>)
        : d_v ? (cut ? k_backward_persistent<CellF, true> : k_backward_persistent<CellF, false>)
              : (cut ? k_backward_persistent<float4, true> : k_backward_persistent<float4, false>);
    int per_sm = 0;
    if ((rc = status_of(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0))))
        return rc;
    if (per_sm < 1) return ART_EINVAL;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(per_sm * g->sms);
    cfg.blockDim = dim3(threads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if ((rc = status_of(cudaLaunchKernelEx(&cfg, kern, A)))) return rc;
    const int unpad_blocks = (int)std::min<long long>((g->ncell + 255) / 256, (long long)g->sms * 16);
    k_unpad_grad<<<unpad_blocks, 256, 0, st>>>(nx, ny, nz, grad_pad, d_dlog_nH0);
    if ((rc = status_of(cudaGetLastError()))) return rc;
    if ((rc = status_of(cudaMemcpyAsync(g->h_stats, g->d_stats, sizeof(DevStats),
                                        cudaMemcpyDeviceToHost, st))))
        return rc;
    g->last_L_in = 0.0;
    for (double v : g->L) g->last_L_in += v;
    g->last_lmax = g->lmax_glob;
    g->destroy_expected = (unsigned long long)ns * (12ull << (2 * g->lmax_glob));
    g->last_kind = 1;
    g->traced = true;
    if (h_stats) return finish_stats(g, h_stats);
    return ART_OK;
}
