// art_internal.h -- host-side grid object shared by the translation units of the library.
#pragma once

#include <vector>

#include <cuda_runtime.h>

#include "art.h"
#include "art_device.cuh"

// A growable array in pinned host memory (copies from it can be captured in a graph).
template <class T>
struct PinnedVec {
    T* data_ = nullptr;
    size_t n_ = 0, cap_ = 0;
    ~PinnedVec() { if (data_) cudaFreeHost(data_); }
    T* data() { return data_; }
    void assign(const T* b, const T* e)
    {
        size_t n = (size_t)(e - b);
        if (n > cap_) {
            if (data_) cudaFreeHost(data_);
            data_ = nullptr;
            cap_ = 0;
            if (cudaMallocHost((void**)&data_, n * sizeof(T)) != cudaSuccess) { data_ = nullptr; n_ = 0; return; }
            cap_ = n;
        }
        for (size_t i = 0; i < n; ++i) data_[i] = b[i];
        n_ = n;
    }
};

struct art_grid {
    int device = 0;
    int sms = 1;
    cudaStream_t stream = nullptr;
    int n[3] = {0, 0, 0};
    long long ncell = 0;
    long long npad = 0;          // cells of the padded layout (sentinel ring around the grid)
    double lo[3] = {0, 0, 0};
    double dx = 1.0;
    const float* nH0 = nullptr;  // borrowed
    const float* nH = nullptr;   // borrowed, may be NULL
    std::vector<double> pos, L;  // host copies of the sources
    std::vector<double> Ln;      // non-ionizing luminosities (two-bin traces)
    bool two_bin = false;
    float2* d_chi2 = nullptr;    // {chi_i, chi_n} per cell length (two-bin traces, padded)
    float* d_srcLn = nullptr;    // base-ray non-ionizing luminosity per source
    size_t srcLn_cap = 0;
    std::vector<float> h_Ln_stage;
    PinnedVec<float> h_srcLn_pin;
    bool buf_2bin[art::kNL] = {};
    std::vector<int> src_lmax;

    // device buffers owned by the grid
    float* d_chi = nullptr;      // opacity per cell length (padded layout)
    float4* d_acc = nullptr;     // per-cell accumulator (padded layout); the reverse sweep
                                 // sums its gradient in the first npad floats
    art::SrcDev* d_src = nullptr;
    size_t src_cap = 0;
    art::LevelInfo* d_levels = nullptr;
    art::Sched* d_sched = nullptr;
    art::DevStats* d_stats = nullptr;
    art::DevStats* h_stats = nullptr;  // pinned

    float4* dir[art::kNL] = {};     // per level: 3 float4 per pixel (n and 1/n as df)
    bool dir_built[art::kNL] = {};
    bool dir_rotate = false;
    double dir_rot[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};

    art::RayBuf buf[art::kNL] = {};
    unsigned long long buf_cap[art::kNL] = {};      // allocated rays per level
    unsigned long long buf_cap_req[art::kNL] = {};
    bool buf_adj[art::kNL] = {};                     // adjoint arrays allocated

    // adjoint: source luminosities and a dL buffer for callers that pass none
    float* d_srcL = nullptr;
    float4* d_rec = nullptr;     // per-cell {chi, chi_H, w, 0} of the reverse sweep (padded)
    art::CellF* d_recf = nullptr;  // the same with the force weight (loss with a force term)
    art::CellW* d_recw = nullptr;  // {chi, w} per cell (loss without dust or force term)
    double* d_dL_scratch = nullptr;
    size_t srcL_cap = 0;
    std::vector<float> h_srcL;

    // what the device copies of the source table and level constants were built from
    art::LevelInfo* h_levels = nullptr;          // pinned staging of the level constants
    PinnedVec<art::SrcDev> h_src_stage;          // pinned staging of the source table
    unsigned long long src_version = 0;
    unsigned long long prep_version = 0;
    bool prep_valid = false, prep_adjoint = false, prep_two_bin = false;
    int prep_level0 = -1, prep_level_max = -2, prep_schedule = -1;
    double prep_m_ray = 0.0;
    long long prep_qcap = -1;

    int lmax_glob = 0;
    int last_lmax = 0;
    int last_kind = 0;  // 0 forward, 1 backward
    double last_L_in = 0.0;
    double last_Ln_in = 0.0;
    bool last_two_bin = false;
    unsigned long long destroy_expected = 0;
    bool traced = false;
};

namespace art {
int check_params(const art_params* p);
int ensure_directions(art_grid* g, const art_params* p, int lfrom, int lto);
int run_opacity(art_grid* g, const art_params* p, bool two_bin);
double rmax_cells(double m_ray, int level);
int prepare_trace(art_grid* g, const art_params* p, bool adjoint);
TraceArgs make_args(art_grid* g, const art_params* p);
int finish_stats(art_grid* g, art_stats* out);
}  // namespace art
