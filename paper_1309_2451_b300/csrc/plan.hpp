// plan.hpp -- host-side state of a ctap plan (internal to libctap).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/ctap.h"
#include "kernels.cuh"

namespace ctap {

struct Event2 {
    cudaEvent_t a, b;
    int kind;
};

// kinetic (and separable-potential) factor tables for one (dt, mode)
struct TabSet {
    double dt;
    int imag;
    void *kin;
    void *sep;
    bool sep_valid;
    void *kin_xy = nullptr;        // real time: (kx, ky) rotations [ny][nx], plan element type (packed complex64 and double-float three-stage Z passes)
};

// an instantiated CUDA graph of one ctap_step call
struct StepGraph {
    void *psi;
    int n;
    double dt;
    int imag;
    cudaGraphExec_t exec;
    long long launches;
    long long uses;
};

struct PlanState {
    // grid
    int nx, ny, nz;
    double box[6];
    ctap_dtype dtype;
    cudaStream_t stream;
    int esize;
    long long N;                   // points of all replicas (batch * Nrep)
    long long Nrep;                // points of one replica
    int batch = 1;                 // independent replicas in one psi
    double dV;
    Geom geom;
    int timeout_ms = 60000;
    bool force_generic = false;    // CTAP_FORCE_GENERIC=1 at plan creation
    bool no_ring = false;          // CTAP_NO_RING=1: one-tile-per-CTA Z pass only
    bool no_packed = false;        // CTAP_NO_PACKED=1: scalar persistent passes instead of packed
    bool fast_xy = false, fast_z = false;
    double vmax = 0.0;             // max |V| over the grid (small-angle kick test)

    // FP64-generated tables on the device (Lift<float> or Lift<double>)
    void *d_tw = nullptr;          // Stockham + cross twiddles
    double *d_k2h = nullptr;       // k^2/2 per axis (FP64)
    std::vector<TabSet> tabsets;   // small cache (adjoint alternates dt and -dt)

    // potential
    int vform = VF_NONE;
    std::vector<double> h_V;       // dense (host copy)
    std::vector<double> h_vsep;    // separable: nx | ny | nz
    std::vector<double> h_g, h_H;  // product
    void *d_Vd = nullptr;          // dense, plan precision
    void *d_g = nullptr;           // product g, plan precision
    void *d_H = nullptr;           // product H, plan precision
    std::vector<double> h_vz;      // product form: additive Vz(z), empty if none
    void *d_vz = nullptr;          // Vz, plan precision
    double *d_vz64 = nullptr;      // Vz, FP64 (observables)
    double *d_g64 = nullptr, *d_H64 = nullptr, *d_vsep64 = nullptr;

    // guides (population regions and adjoint data)
    bool have_regions = false;
    double hw = 1.5;
    double *d_xc = nullptr;        // [3][nz]
    std::vector<double> h_xc;
    bool have_guides = false;
    double V0 = 0.0, s = 1.0;
    std::vector<double> h_x1, h_x3;
    double *d_D1 = nullptr, *d_D3 = nullptr;   // dV/dx_j / g(y), [nz][nx]
    bool have_spline = false;
    std::vector<double> knots, c12, c23;
    std::vector<double> basis;     // [nknots][nz]

    // scratch
    double *d_partials = nullptr;
    size_t n_partials = 0;
    double *d_red = nullptr;       // 8 doubles
    double *d_scale = nullptr;     // 1 double
    void *d_work = nullptr;        // one psi, lazily (observables)
    double *d_dens = nullptr;      // nz x nx doubles, lazily (density_xz)

    // accounting
    long long launches = 0;
    bool profiling = false;
    std::vector<Event2> events;
    size_t events_used = 0;
    long long prof_counts[3] = {0, 0, 0};
    double prof_ms[3] = {0, 0, 0};

    // CUDA graphs of repeated ctap_step calls (non-default streams only)
    bool graphs = true;
    std::vector<StepGraph> step_graphs;

    std::string err;
};

// tables.cpp
void build_geometry(PlanState &p, int emax, int maxv);   // throws std::runtime_error
void build_twiddles(PlanState &p, std::vector<unsigned char> &host, int maxv);
void build_kinetic(const PlanState &p, double dt, int imag, std::vector<unsigned char> &host);
// real time, complex64: Lift<float> of exp(-i (kx^2 + ky^2) dt/2), [ny][nx]
void build_kinetic_xy(const PlanState &p, double dt, std::vector<unsigned char> &host);
void build_k2h(const PlanState &p, std::vector<double> &host);
void build_separable(const PlanState &p, double dt, int imag, std::vector<unsigned char> &host);
void natural_spline_basis(const std::vector<double> &knots, const std::vector<double> &z,
                          std::vector<double> &B);
double grid_point(int i, int n, double lo, double hi);

}  // namespace ctap

struct ctap_plan {
    ctap::PlanState st;
};
