// art_shard.cu -- splitting one trace over several GPUs by source (new; the paper's MPI
// version decomposes the domain and passes rays between ranks instead, Sec. 2.2).
//
// Sources are independent and their deposits add (Sec. 2.1: several sources are handled by
// summing over the rays of every source), so N ranks can each trace a disjoint subset of the
// sources over a replicated density field and sum their per-cell outputs with one
// all-reduce. The rank with the most work sets the time, so the subsets are chosen by a
// per-source work estimate:
//   * art_estimate_work walks a coarse HEALPix set of rays from every source, without
//     splitting, to where the trace would retire them (tau > tau_max, the d_max cutoff or the
//     grid boundary), and turns the reach D of each coarse ray into the crossings of the rays
//     that cover its solid angle in the full trace;
//   * art_partition_sources assigns sources to ranks by longest-processing-time-first
//     greedy (each source, largest estimate first, to the least-loaded rank), whose largest
//     load is at most 4/3 of the best possible.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "art.h"
#include "art_internal.h"

using namespace art;

namespace {

// Reach of the coarse ray (source s, pixel p of the coarse level) in cell units: where the
// walk from the source ends at tau > tau_max, at the cutoff radius dmax or at the grid
// boundary. No deposits and no splits. Every step crosses at least one face, so a walk
// ends within nx + ny + nz + 2 steps.
__global__ void k_reach(int nx, int ny, int nz, const float* __restrict__ chi,
                        const SrcDev* __restrict__ src, int nsrc, const float4* __restrict__ dir,
                        unsigned npix, float tau_max, df dmax, float* __restrict__ reach)
{
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= (unsigned long long)nsrc * npix) return;
    const unsigned s = (unsigned)(i / npix), p = (unsigned)(i - (unsigned long long)s * npix);
    const float4 sh = __ldg(&src[s].hi), sl = __ldg(&src[s].lo);
    const float4 e0 = __ldg(dir + 3ull * p), e1 = __ldg(dir + 3ull * p + 1), e2 = __ldg(dir + 3ull * p + 2);
    const df u[3] = {{sh.x, sl.x}, {sh.y, sl.y}, {sh.z, sl.z}};
    const df n[3] = {{e0.x, e0.w}, {e0.y, e1.x}, {e0.z, e1.y}};
    const df inv[3] = {{e1.z, e2.y}, {e1.w, e2.z}, {e2.x, e2.w}};
    WalkT<float> W;
    if (!walk_start(W, nx, ny, nz, u, n, inv, df{0.f, 0.f})) {
        reach[i] = 0.f;
        return;
    }
    W.L = 0.f;
    W.Lc = 0.f;
    W.tau = 0.f;
    W.cell = __ldg(chi + W.idx);
    float r = 0.f;
    const int bound = nx + ny + nz + 2;
    for (int k = 0; k < bound; ++k) {
        const df before = W.tc;
        const StepOut o = walk_step<true>(W, true, dmax, chi, tau_max);
        if (o.ev == EV_NONE) continue;
        // an exit is seen one step late, in the sentinel cell: the ray left at `before`
        r = o.ev == EV_EXIT ? before.hi : fminf(W.tc.hi, dmax.hi);
        break;
    }
    reach[i] = r;
}

}  // namespace

extern "C" {

int art_estimate_work(art_grid* g, const art_params* p, double* h_work)
{
    if (!g || !h_work) return ART_EINVAL;
    int rc = check_params(p);
    if (rc) return rc;
    const int ns = (int)g->L.size();
    if (ns == 0) return ART_ESTATE;
    // coarse level: 192 rays per source (or the base level when that is coarser)
    const int le = std::min(p->level0, 2);
    const unsigned npix = 12u << (2 * le);
    // source table (positions in cell units as double-floats)
    std::vector<SrcDev> hs(ns);
    for (int s = 0; s < ns; ++s) {
        float h[3], lo[3];
        for (int a = 0; a < 3; ++a) {
            const double u = (g->pos[3 * s + a] - g->lo[a]) / g->dx;
            h[a] = (float)u;
            lo[a] = (float)(u - (double)h[a]);
        }
        hs[s].hi = make_float4(h[0], h[1], h[2], 0.f);
        hs[s].lo = make_float4(lo[0], lo[1], lo[2], 0.f);
    }
    if ((rc = ensure_directions(g, p, le, le))) return rc;
    if ((rc = run_opacity(g, p, false))) return rc;
    SrcDev* d_src = nullptr;
    float* d_reach = nullptr;
    const size_t nray = (size_t)ns * npix;
    cudaError_t e = cudaMalloc((void**)&d_src, sizeof(SrcDev) * ns);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_reach, sizeof(float) * nray);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_src, hs.data(), sizeof(SrcDev) * ns, cudaMemcpyHostToDevice, g->stream);
    std::vector<float> reach(nray);
    if (e == cudaSuccess) {
        df dmax;
        const double dm = p->d_max > 0.0 ? p->d_max / g->dx : 1.0e30;
        dmax.hi = (float)dm;
        dmax.lo = (float)(dm - (double)dmax.hi);
        k_reach<<<(unsigned)((nray + 255) / 256), 256, 0, g->stream>>>(
            g->n[0], g->n[1], g->n[2], g->d_chi, d_src, ns, g->dir[le], npix, (float)p->tau_max,
            dmax, d_reach);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(reach.data(), d_reach, sizeof(float) * nray, cudaMemcpyDeviceToHost,
                            g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (d_src) cudaFree(d_src);
    if (d_reach) cudaFree(d_reach);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ART_ENOMEM : ART_ECUDA;
    // Crossings of the rays that cover a coarse ray's solid angle Omega = 4 pi / npix out to
    // its reach D: inside r0 = r_max(l0) the N0 / npix base rays each cross about 1.5 cells
    // per cell of path (the mean of |n_x| + |n_y| + |n_z| over the sphere); beyond it the
    // splitting keeps m_ray to 4 m_ray rays per cell face, about m_ray Omega r^2 rays at
    // radius r on average over a level, hence ~ m_ray Omega (D^3 - r0^3) crossings.
    const double r0 = rmax_cells(p->m_ray, p->level0);
    const double base = (double)(12u << (2 * p->level0)) / (double)npix;
    const double omega = 4.0 * M_PI / (double)npix;
    for (int s = 0; s < ns; ++s) {
        double w = 0.0;
        for (unsigned q = 0; q < npix; ++q) {
            const double D = reach[(size_t)s * npix + q];
            w += 1.5 * base * std::min(D, r0);
            if (D > r0) w += p->m_ray * omega * (D * D * D - r0 * r0 * r0);
        }
        h_work[s] = w;
    }
    return ART_OK;
}

int art_partition_sources(int n, const double* h_work, int nranks, int* h_rank, double* h_load)
{
    if (n < 0 || nranks < 1 || (n > 0 && (!h_work || !h_rank))) return ART_EINVAL;
    for (int s = 0; s < n; ++s)
        if (!(h_work[s] >= 0.0) || !std::isfinite(h_work[s])) return ART_EINVAL;
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    // largest estimate first; equal estimates by source index, so every rank computes the
    // same assignment
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return h_work[a] > h_work[b]; });
    std::vector<double> load(nranks, 0.0);
    for (int s : order) {
        int best = 0;
        for (int r = 1; r < nranks; ++r)
            if (load[r] < load[best]) best = r;
        h_rank[s] = best;
        load[best] += h_work[s];
    }
    if (h_load) std::memcpy(h_load, load.data(), sizeof(double) * nranks);
    return ART_OK;
}

}  // extern "C"
