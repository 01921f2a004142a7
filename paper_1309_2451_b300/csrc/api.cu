// api.cu -- the C ABI of libctap (declared in include/ctap.h): plan life
// cycle, potentials, the split-step driver (Sec. IV), observables (Sec. V,
// Fig. 4) and the adjoint gradient driver.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "packed_passes.cuh"
#include "plan.hpp"

using namespace ctap;

namespace {

// ----------------------------------------------------- host fault injection
// CTAP_FAULT_INJECT=alloc:N or launch:N makes the N-th device allocation or
// kernel launch (counted over the process, from 1) fail before it touches
// the GPU.  For exercising error paths only.
struct FaultInjector {
    long long alloc_at = -1, launch_at = -1;
    long long allocs = 0, launches = 0;
    bool parsed = false;
    void parse()
    {
        if (parsed) return;
        parsed = true;
        const char *e = std::getenv("CTAP_FAULT_INJECT");
        if (!e) return;
        if (std::strncmp(e, "alloc:", 6) == 0) alloc_at = std::atoll(e + 6);
        if (std::strncmp(e, "launch:", 7) == 0) launch_at = std::atoll(e + 7);
    }
    bool alloc_fails() { parse(); return ++allocs == alloc_at; }
    bool launch_fails() { parse(); return ++launches == launch_at; }
} g_fault;

ctap_status fail(PlanState &st, ctap_status s, const std::string &msg)
{
    st.err = msg;
    return s;
}

ctap_status cuda_fail(PlanState &st, cudaError_t e, const char *what)
{
    st.err = std::string(what) + ": " + cudaGetErrorString(e);
    return CTAP_ERR_CUDA;
}

ctap_status dev_alloc(PlanState &st, void **p, size_t bytes)
{
    *p = nullptr;
    if (g_fault.alloc_fails()) return fail(st, CTAP_ERR_OOM, "injected allocation failure");
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(st, CTAP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return CTAP_OK;
}

void dev_free(void *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}
template <class U> void dev_free_t(U *&p)
{
    void *q = p;
    dev_free(q);
    p = nullptr;
}

// host-side wait with a deadline (no device-side spinning anywhere)
ctap_status wait_stream(PlanState &st, int timeout_ms)
{
    const int tmo = timeout_ms > 0 ? timeout_ms : st.timeout_ms;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(st.stream);
        if (e == cudaSuccess) return CTAP_OK;
        if (e != cudaErrorNotReady) return cuda_fail(st, e, "stream");
        const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(
            std::chrono::steady_clock::now() - t0);
        if (el.count() > tmo) return fail(st, CTAP_ERR_TIMEOUT, "stream did not finish in time");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

ctap_status upload(PlanState &st, void **dptr, size_t *have, const void *src, size_t bytes)
{
    if (*dptr == nullptr || (have && *have < bytes)) {
        dev_free(*dptr);
        ctap_status s = dev_alloc(st, dptr, bytes);
        if (s != CTAP_OK) return s;
        if (have) *have = bytes;
    }
    cudaError_t e = cudaMemcpyAsync(*dptr, src, bytes, cudaMemcpyHostToDevice, st.stream);
    if (e != cudaSuccess) return cuda_fail(st, e, "upload");
    return wait_stream(st, 0);   // host source is released by the caller
}

// ------------------------------------------------------------ launch hooks
int prof_begin(PlanState &st, int kind)
{
    if (!st.profiling) return -1;
    if (st.events_used == st.events.size()) {
        Event2 ev{};
        cudaEventCreate(&ev.a);
        cudaEventCreate(&ev.b);
        st.events.push_back(ev);
    }
    Event2 &ev = st.events[st.events_used];
    ev.kind = kind;
    cudaEventRecord(ev.a, st.stream);
    return (int)st.events_used++;
}

void prof_end(PlanState &st, int idx)
{
    if (idx >= 0) cudaEventRecord(st.events[idx].b, st.stream);
}

ctap_status pre_launch(PlanState &st)
{
    if (g_fault.launch_fails()) return fail(st, CTAP_ERR_CUDA, "injected launch failure");
    return CTAP_OK;
}

ctap_status post_launch(PlanState &st, const char *what)
{
    ++st.launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(st, e, what);
    return CTAP_OK;
}

#define CTAP_TRY(x)                              \
    do {                                         \
        ctap_status _s = (x);                    \
        if (_s != CTAP_OK) return _s;            \
    } while (0)

// ----------------------------------------------------------- table caches
// Captured step graphs hold device pointers to tables and potentials: drop
// them before any of those is freed or replaced.
void drop_graphs(PlanState &st)
{
    if (!st.step_graphs.empty()) cudaStreamSynchronize(st.stream);
    for (auto &g : st.step_graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    st.step_graphs.clear();
}

void drop_caches(PlanState &st)
{
    drop_graphs(st);
    for (auto &t : st.tabsets) {
        dev_free(t.kin);
        dev_free(t.sep);
        dev_free(t.kin_xy);
    }
    st.tabsets.clear();
}

void invalidate_sep(PlanState &st)
{
    drop_graphs(st);
    for (auto &t : st.tabsets) t.sep_valid = false;
}

// the packed persistent Z pass applies to this plan's steady real-time steps
bool packed_z_on(const PlanState &st)
{
    return st.fast_z && !st.no_ring && !st.no_packed && st.dtype == CTAP_C64 &&
           packed_z_supported(st.geom);
}

ctap_status get_tables(PlanState &st, double dt, int imag, TabSet **out)
{
    std::vector<TabSet> &c = st.tabsets;
    TabSet *hit = nullptr;
    for (auto &t : c)
        if (t.dt == dt && t.imag == imag) hit = &t;
    if (!hit || (st.vform == VF_SEPARABLE && !hit->sep_valid)) drop_graphs(st);
    if (!hit) {
        if (c.size() >= 4) {
            dev_free(c.front().kin);
            dev_free(c.front().sep);
            dev_free(c.front().kin_xy);
            c.erase(c.begin());
        }
        c.push_back(TabSet{dt, imag, nullptr, nullptr, false});
        hit = &c.back();
        std::vector<unsigned char> h;
        build_kinetic(st, dt, imag, h);
        CTAP_TRY(upload(st, &hit->kin, nullptr, h.data(), h.size()));
        // the (kx, ky) kinetic rotation of each column as one table entry:
        // the packed complex64 Z pass and the double-float three-stage one
        const bool df_z3 = st.dtype == CTAP_C128_DF && st.fast_z && st.nz == 1024;
        if ((packed_z_on(st) || df_z3) && !imag) {
            build_kinetic_xy(st, dt, h);
            CTAP_TRY(upload(st, &hit->kin_xy, nullptr, h.data(), h.size()));
        }
    }
    if (st.vform == VF_SEPARABLE && !hit->sep_valid) {
        std::vector<unsigned char> h;
        build_separable(st, dt, imag, h);
        dev_free(hit->sep);
        CTAP_TRY(upload(st, &hit->sep, nullptr, h.data(), h.size()));
        hit->sep_valid = true;
    }
    *out = hit;
    return CTAP_OK;
}

// ----------------------------------------------------------- pass drivers
template <class T> XYArgs<T> xy_args(PlanState &st, const TabSet *ts, double dt, int imag)
{
    XYArgs<T> a{};
    a.g = st.geom;
    a.tw = reinterpret_cast<const Lift<T> *>(st.d_tw);
    a.k.form = st.vform == VF_SEPARABLE ? VF_SEPARABLE
                                        : (st.vform == VF_DENSE ? VF_DENSE : VF_PRODUCT);
    a.k.imag = imag;
    a.k.Vd = reinterpret_cast<const T *>(st.d_Vd);
    a.k.g = reinterpret_cast<const T *>(st.d_g);
    a.k.H = reinterpret_cast<const T *>(st.d_H);
    a.k.vz = reinterpret_cast<const T *>(st.d_vz);
    if (ts && ts->sep) {
        const size_t n = (size_t)(st.nx + st.ny + st.nz);
        a.k.sep_half = reinterpret_cast<const Lift<T> *>(ts->sep);
        a.k.sep_full = reinterpret_cast<const Lift<T> *>(ts->sep) + n;
    }
    a.k.tau_half = (T)(0.5 * dt);
    a.k.tau_full = (T)dt;
    a.rd.Vsep = st.d_vsep64;
    a.rd.g64 = st.d_g64;
    a.rd.H64 = st.d_H64;
    a.rd.vz64 = st.d_vz64;
    a.rd.xc = st.have_regions ? st.d_xc : nullptr;
    a.rd.hw = st.hw;
    a.rd.k2h = st.d_k2h;
    a.vform_obs = st.vform;
    a.partials = st.d_partials;
    // short kick series: |V| dt <= 0.5 (FP32 series) or <= 0.1 (FP64 series);
    // complex64 also has a shorter series for |V| dt <= 0.16
    const double vdt = st.vmax * std::fabs(dt);
    a.small_angle = (vdt <= (sizeof(T) == 4 ? 0.5 : 0.1)) ? 1 : 0;
    if (std::is_same<T, float>::value && vdt <= 0.16) a.small_angle = 2;
    a.ring = st.no_ring ? 0 : 1;
    return a;
}

template <class T> ZArgs<T> z_args(PlanState &st, const TabSet *ts, int imag)
{
    ZArgs<T> a{};
    a.g = st.geom;
    a.tw = reinterpret_cast<const Lift<T> *>(st.d_tw);
    a.kin = ts ? reinterpret_cast<const Lift<T> *>(ts->kin) : nullptr;
    a.kin_xy = ts ? ts->kin_xy : nullptr;
    a.imag = imag;
    a.inv_n = (T)(1.0 / (double)st.Nrep);      // transforms act on one replica
    a.k2h = st.d_k2h;
    a.partials = st.d_partials;
    a.ring = st.no_ring ? 0 : 1;
    return a;
}

template <class T> ctap_status go_xy(PlanState &st, const XYArgs<T> &a)
{
    CTAP_TRY(pre_launch(st));
    // kind 0: the steady XY pass; prologue/epilogue/observe variants count as 2
    const bool steady = (a.flags & (XY_IN_MIXED | XY_OUT_MIXED)) == (XY_IN_MIXED | XY_OUT_MIXED);
    int ev = prof_begin(st, steady ? 0 : 2);
    bool done = false;
    // the fast XY pass moves two values per 16-byte access
    const bool aligned = ((reinterpret_cast<uintptr_t>(a.src) | reinterpret_cast<uintptr_t>(a.dst)) & 15) == 0;
    if constexpr (std::is_same<T, float>::value) {
        if (st.fast_xy && aligned && !st.no_packed) done = launch_xy_packed(a, st.stream);
    }
    if (!done && st.fast_xy && aligned) done = launch_xy_fast(a, st.stream);
    if (!done) launch_xy<T>(a, st.stream);
    prof_end(st, ev);
    return post_launch(st, "xy pass");
}

template <class T> ctap_status go_z(PlanState &st, const ZArgs<T> &a)
{
    CTAP_TRY(pre_launch(st));
    int ev = prof_begin(st, 1);
    bool done = false;
    // the fast Z pass moves two columns per 16-byte access
    const bool aligned = ((reinterpret_cast<uintptr_t>(a.src) | reinterpret_cast<uintptr_t>(a.dst)) & 15) == 0;
    if constexpr (std::is_same<T, float>::value) {
        if (st.fast_z && aligned && !st.no_packed) done = launch_z_packed(a, st.stream);
    }
    if (!done && st.fast_z && aligned) done = launch_z_fast(a, st.stream);
    if (!done) launch_z<T>(a, st.stream);
    prof_end(st, ev);
    return post_launch(st, "z pass");
}

template <class F> ctap_status go_other(PlanState &st, const char *what, F f)
{
    CTAP_TRY(pre_launch(st));
    int ev = prof_begin(st, 2);
    f();
    prof_end(st, ev);
    return post_launch(st, what);
}

// K/2 V K/2 steps in real time: the kinetic halves of consecutive steps
// merge, so the pass sequence is XY (forward only), Z (K/2), n times
// [XY (inverse, full V, forward), Z (K, the last one K/2)], XY (inverse only).
template <class T> ctap_status run_steps_kvk(PlanState &st, Cx<T> *psi, int n, double dt)
{
    TabSet *ts = nullptr;
    CTAP_TRY(get_tables(st, dt, 0, &ts));
    XYArgs<T> xa = xy_args<T>(st, ts, dt, 0);
    ZArgs<T> za = z_args<T>(st, ts, 0);         // kinetic pointers copied before the
    TabSet *th = nullptr;                       // cache may move its entries
    CTAP_TRY(get_tables(st, 0.5 * dt, 0, &th));
    ZArgs<T> zh = z_args<T>(st, th, 0);
    xa.src = za.src = zh.src = psi;
    xa.dst = za.dst = zh.dst = psi;
    xa.flags = XY_OUT_MIXED;
    CTAP_TRY(go_xy<T>(st, xa));
    CTAP_TRY(go_z<T>(st, zh));
    for (int s = 0; s < n; ++s) {
        xa.flags = XY_IN_MIXED | XY_KICK_FULL | XY_OUT_MIXED;
        CTAP_TRY(go_xy<T>(st, xa));
        CTAP_TRY(go_z<T>(st, s + 1 < n ? za : zh));
    }
    xa.flags = XY_IN_MIXED;
    return go_xy<T>(st, xa);
}

// nsteps Strang steps on psi (device, natural layout in and out); mode is a
// ctap_time value
template <class T> ctap_status run_steps(PlanState &st, Cx<T> *psi, int n, double dt, int mode)
{
    if (n <= 0) return CTAP_OK;
    if (mode == CTAP_REAL_KVK) return run_steps_kvk<T>(st, psi, n, dt);
    const int imag = mode == CTAP_IMAG ? 1 : 0;
    TabSet *ts = nullptr;
    CTAP_TRY(get_tables(st, dt, imag, &ts));
    XYArgs<T> xa = xy_args<T>(st, ts, dt, imag);
    ZArgs<T> za = z_args<T>(st, ts, imag);
    xa.src = psi;
    xa.dst = psi;
    za.src = psi;
    za.dst = psi;
    const int nxy = xy_grid(st.geom);

    xa.flags = XY_KICK_HALF | XY_OUT_MIXED;                       // V/2, forward x,y
    CTAP_TRY(go_xy<T>(st, xa));
    for (int s = 0; s < n; ++s) {
        za.scale = (imag && s > 0) ? st.d_scale : nullptr;
        CTAP_TRY(go_z<T>(st, za));                                // cross, F_z, K, I_z
        if (s + 1 < n) {
            if (imag) {
                xa.flags = XY_IN_MIXED | XY_KICK_SPLIT | XY_RED_NORM | XY_OUT_MIXED;
                CTAP_TRY(go_xy<T>(st, xa));
                CTAP_TRY(go_other(st, "norm", [&] {
                    launch_norm_scale(st.d_partials, nxy, st.dV, st.d_scale, st.stream);
                }));
            } else {
                xa.flags = XY_IN_MIXED | XY_KICK_FULL | XY_OUT_MIXED;   // V/2 + V/2 merged
                CTAP_TRY(go_xy<T>(st, xa));
            }
        }
    }
    xa.flags = XY_IN_MIXED | XY_KICK_HALF | (imag ? XY_RED_NORM : 0);  // inverse x,y, V/2
    CTAP_TRY(go_xy<T>(st, xa));
    if (imag) {
        CTAP_TRY(go_other(st, "norm", [&] {
            launch_norm_scale(st.d_partials, nxy, st.dV, st.d_scale, st.stream);
        }));
        CTAP_TRY(go_other(st, "scale", [&] { launch_scale<T>(psi, st.N, st.d_scale, st.stream); }));
    }
    return CTAP_OK;
}

// Replay a captured graph for a repeated (psi, n, dt, mode) call.  The first
// call runs eagerly; the second captures the launch sequence once (tables are
// uploaded before capture begins) and replays it; later calls replay.

template <class T> ctap_status step_maybe_graph(PlanState &st, Cx<T> *psi, int n, double dt, int mode)
{
    const int imag = mode;                      // graph key: the full ctap_time mode
    const bool usable = st.graphs && st.stream != nullptr && !st.profiling &&
                        !std::getenv("CTAP_FAULT_INJECT") && n > 0;
    if (!usable) return run_steps<T>(st, psi, n, dt, imag);
    for (auto &g : st.step_graphs) {
        if (g.psi == psi && g.n == n && g.dt == dt && g.imag == imag) {
            if (g.exec) {
                cudaError_t e = cudaGraphLaunch(g.exec, st.stream);
                if (e != cudaSuccess) return cuda_fail(st, e, "graph launch");
                st.launches += g.launches;
                return CTAP_OK;
            }
            // second sighting: capture (tables are built by the eager first call)
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(st.stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(st, e, "begin capture");
            const long long l0 = st.launches;
            ctap_status s = run_steps<T>(st, psi, n, dt, imag);
            cudaError_t e2 = cudaStreamEndCapture(st.stream, &graph);
            if (s != CTAP_OK) {
                if (graph) cudaGraphDestroy(graph);
                return s;
            }
            if (e2 != cudaSuccess) return cuda_fail(st, e2, "end capture");
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(st, e, "graph instantiate");
            g.exec = exec;
            g.launches = st.launches - l0;
            st.launches = l0;
            e = cudaGraphLaunch(exec, st.stream);
            if (e != cudaSuccess) return cuda_fail(st, e, "graph launch");
            st.launches += g.launches;
            return CTAP_OK;
        }
    }
    if (st.step_graphs.size() >= 8) {
        if (st.step_graphs.front().exec) cudaGraphExecDestroy(st.step_graphs.front().exec);
        st.step_graphs.erase(st.step_graphs.begin());
    }
    st.step_graphs.push_back(StepGraph{psi, n, dt, imag, nullptr, 0, 0});
    return run_steps<T>(st, psi, n, dt, imag);
}

ctap_status ensure_work(PlanState &st)
{
    if (st.d_work) return CTAP_OK;
    return dev_alloc(st, &st.d_work, (size_t)st.N * st.esize);
}

// raw FP64 sums: [s2, sV, p1, p2, p3, sk]
template <class T> ctap_status observe_raw(PlanState &st, const Cx<T> *psi, double *raw)
{
    CTAP_TRY(ensure_work(st));
    XYArgs<T> xa = xy_args<T>(st, nullptr, 0.0, 0);
    ZArgs<T> za = z_args<T>(st, nullptr, 0);
    const int nxy = xy_grid(st.geom), nz_ = z_grid(st.geom);
    xa.src = psi;
    xa.dst = reinterpret_cast<Cx<T> *>(st.d_work);
    xa.flags = XY_RED_OBS | XY_OUT_MIXED;
    xa.partials = st.d_partials;
    CTAP_TRY(go_xy<T>(st, xa));
    // per-CTA partials are replica-major in both passes: one fixed-order sum per replica
    const int B = st.batch, nxy_r = nxy / B, nz_r = nz_ / B;
    CTAP_TRY(go_other(st, "reduce", [&] {
        for (int b = 0; b < B; ++b)
            launch_reduce(st.d_partials + (size_t)5 * nxy_r * b, nxy_r, 5, st.d_red + 8 * b,
                          st.stream);
    }));
    za.src = reinterpret_cast<const Cx<T> *>(st.d_work);
    za.dst = nullptr;
    za.observe = 1;
    za.partials = st.d_partials + (size_t)5 * nxy;
    CTAP_TRY(go_z<T>(st, za));
    CTAP_TRY(go_other(st, "reduce", [&] {
        for (int b = 0; b < B; ++b)
            launch_reduce(st.d_partials + (size_t)5 * nxy + (size_t)nz_r * b, nz_r, 1,
                          st.d_red + 8 * b + 5, st.stream);
    }));
    cudaError_t e = cudaMemcpyAsync(raw, st.d_red, 8 * (size_t)B * sizeof(double),
                                    cudaMemcpyDeviceToHost, st.stream);
    if (e != cudaSuccess) return cuda_fail(st, e, "observables copy");
    return wait_stream(st, 0);
}

ctap_status finish_observables(PlanState &st, const double *raw, double *out)
{
    const double s2 = raw[0];
    out[0] = s2 * st.dV;
    out[1] = s2 > 0 ? raw[5] / ((double)st.Nrep * s2) : 0.0;
    out[2] = s2 > 0 ? raw[1] / s2 : 0.0;
    for (int j = 0; j < 3; ++j) out[3 + j] = st.have_regions ? raw[2 + j] * st.dV : 0.0;
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(out[i])) return fail(st, CTAP_ERR_NONFINITE, "non-finite observable");
    return CTAP_OK;
}

// ------------------------------------------------------------- adjoint
// Recompute the states of one checkpoint segment: from psi_{n0} (natural,
// copied into `work`), L steps; the steady XY pass writes psi_{n0+i} to
// states[i] between its two half-kicks, the last pass writes psi_{n0+L} to
// states[L].  2 L + 1 launches, no copies.
template <class T>
ctap_status record_segment(PlanState &st, Cx<T> *work, int L, double dt, Cx<T> *const *states)
{
    TabSet *ts = nullptr;
    CTAP_TRY(get_tables(st, dt, 0, &ts));
    XYArgs<T> xa = xy_args<T>(st, ts, dt, 0);
    ZArgs<T> za = z_args<T>(st, ts, 0);
    xa.src = xa.dst = work;
    za.src = za.dst = work;
    xa.flags = XY_KICK_HALF | XY_OUT_MIXED;
    CTAP_TRY(go_xy<T>(st, xa));
    for (int s = 0; s < L; ++s) {
        CTAP_TRY(go_z<T>(st, za));
        if (s + 1 < L) {
            xa.flags = XY_IN_MIXED | XY_KICK_SPLIT | XY_STATE_OUT | XY_OUT_MIXED;
            xa.state_out = states[s + 1];
            CTAP_TRY(go_xy<T>(st, xa));
        }
    }
    xa.flags = XY_IN_MIXED | XY_KICK_HALF;
    xa.dst = states[L];
    return go_xy<T>(st, xa);
}

// Sweep lambda back over one segment: lambda_{n1} (natural, in place) ->
// lambda_{n0} with steps of -dt (S(-dt) is the adjoint of S(dt)).  Each XY
// pass adds dt w_m sum Im(conj(lambda_m) psi_m) dV/dx_j to the per-CTA
// partials at the integer step it holds: the first pass at m = n1 (its
// input), the steady passes between their half-kicks, the last pass (only
// when `bottom`) at m = n0.  psi[i] is psi_{n0+i}.
template <class T>
ctap_status lambda_segment(PlanState &st, Cx<T> *lam, int L, double dt, const Cx<T> *const *psi,
                           double coef_top, bool bottom, double coef_bottom, double *acc)
{
    TabSet *ts = nullptr;
    CTAP_TRY(get_tables(st, -dt, 0, &ts));
    XYArgs<T> xa = xy_args<T>(st, ts, -dt, 0);
    ZArgs<T> za = z_args<T>(st, ts, 0);
    xa.src = xa.dst = lam;
    za.src = za.dst = lam;
    xa.gd.g64 = st.d_g64;
    xa.gd.D1 = st.d_D1;
    xa.gd.D3 = st.d_D3;
    xa.gd.acc = acc;
    const double interior = 2.0 * dt * st.dV;
    xa.flags = XY_KICK_HALF | XY_OUT_MIXED | XY_GRAD_PRE;
    xa.gd.psi = psi[L];
    xa.gd.coef = coef_top;
    CTAP_TRY(go_xy<T>(st, xa));
    for (int s = 0; s < L; ++s) {
        CTAP_TRY(go_z<T>(st, za));
        if (s + 1 < L) {
            xa.flags = XY_IN_MIXED | XY_KICK_SPLIT | XY_GRAD | XY_OUT_MIXED;
            xa.gd.psi = psi[L - 1 - s];
            xa.gd.coef = interior;
            CTAP_TRY(go_xy<T>(st, xa));
        }
    }
    xa.flags = XY_IN_MIXED | XY_KICK_HALF | (bottom ? XY_GRAD : 0);
    xa.gd.psi = psi[0];
    xa.gd.coef = coef_bottom;
    return go_xy<T>(st, xa);
}

template <class T>
ctap_status run_adjoint(PlanState &st, const Cx<T> *psi0, int nsteps, double dt, int K, int guide,
                        double *J, double *grad)
{
    const size_t bytes = (size_t)st.N * sizeof(Cx<T>);
    const int nseg = (nsteps + K - 1) / K;
    const int Kseg = std::min(K, nsteps);
    const int nacc = xy_grid(st.geom);
    struct Bufs {
        void *cp = nullptr, *seg = nullptr, *work = nullptr, *lam = nullptr, *acc = nullptr;
        ~Bufs()
        {
            dev_free(cp);
            dev_free(seg);
            dev_free(work);
            dev_free(lam);
            dev_free(acc);
        }
    } b;
    // nseg checkpoints + one segment of Kseg states + two working states:
    // refuse before allocating when that cannot fit in the free device memory
    {
        size_t freeb = 0, totalb = 0;
        const double need = (double)bytes * (double)(nseg + Kseg + 2) + 16.0 * nacc;
        if (cudaMemGetInfo(&freeb, &totalb) == cudaSuccess && need > 0.95 * (double)freeb) {
            char msg[160];
            std::snprintf(msg, sizeof msg,
                          "adjoint needs %.1f GB of checkpoints and segment states, %.1f GB "
                          "free; use a larger K or fewer steps",
                          need / 1e9, (double)freeb / 1e9);
            return fail(st, CTAP_ERR_OOM, msg);
        }
    }
    CTAP_TRY(dev_alloc(st, &b.cp, bytes * nseg));
    CTAP_TRY(dev_alloc(st, &b.seg, bytes * Kseg));
    CTAP_TRY(dev_alloc(st, &b.work, bytes));
    CTAP_TRY(dev_alloc(st, &b.lam, bytes));
    CTAP_TRY(dev_alloc(st, &b.acc, sizeof(double) * 2 * nacc));
    auto at = [&](void *base, size_t i) {
        return reinterpret_cast<Cx<T> *>(static_cast<char *>(base) + i * bytes);
    };
    auto copy = [&](Cx<T> *dst, const Cx<T> *src) -> ctap_status {
        cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st.stream);
        return e == cudaSuccess ? CTAP_OK : cuda_fail(st, e, "copy");
    };
    double *acc = static_cast<double *>(b.acc);
    if (cudaMemsetAsync(acc, 0, sizeof(double) * 2 * nacc, st.stream) != cudaSuccess)
        return fail(st, CTAP_ERR_CUDA, "memset");

    // forward sweep with checkpoints psi_{sK}
    Cx<T> *cur = at(b.work, 0);
    CTAP_TRY(copy(cur, psi0));
    for (int s = 0; s < nseg; ++s) {
        CTAP_TRY(copy(at(b.cp, s), cur));
        CTAP_TRY(run_steps<T>(st, cur, std::min(K, nsteps - s * K), dt, 0));
    }
    // J and lambda_N = M psi_N
    Cx<T> *lam = at(b.lam, 0);
    const int nmb = mask_blocks(st.geom);
    CTAP_TRY(go_other(st, "mask", [&] {
        launch_mask<T>(cur, lam, st.geom, st.d_xc + (size_t)(guide - 1) * st.nz, st.hw,
                       st.d_partials, nmb, st.stream);
    }));
    CTAP_TRY(go_other(st, "reduce", [&] { launch_reduce(st.d_partials, nmb, 1, st.d_red, st.stream); }));

    // backward sweep, one checkpoint segment at a time
    std::vector<Cx<T> *> states(Kseg + 1);
    for (int s = nseg - 1; s >= 0; --s) {
        const int n0 = s * K, n1 = std::min((s + 1) * K, nsteps), L = n1 - n0;
        states[0] = at(b.cp, s);
        for (int i = 1; i <= L; ++i) states[i] = at(b.seg, i - 1);
        CTAP_TRY(copy(cur, states[0]));
        CTAP_TRY(record_segment<T>(st, cur, L, dt, states.data()));
        const double wtop = (n1 == nsteps) ? 1.0 : 2.0;
        CTAP_TRY(lambda_segment<T>(st, lam, L, dt, states.data(), dt * wtop * st.dV, s == 0,
                                   dt * st.dV, acc));
    }
    std::vector<double> hacc(2 * (size_t)nacc);
    double hJ = 0.0;
    if (cudaMemcpyAsync(hacc.data(), acc, sizeof(double) * 2 * nacc, cudaMemcpyDeviceToHost,
                        st.stream) != cudaSuccess ||
        cudaMemcpyAsync(&hJ, st.d_red, sizeof(double), cudaMemcpyDeviceToHost, st.stream) !=
            cudaSuccess)
        return fail(st, CTAP_ERR_CUDA, "adjoint copy");
    CTAP_TRY(wait_stream(st, 0));
    *J = hJ * st.dV;
    // per-slice sensitivities R_j(z): sum over the row classes of the plane
    const int P = st.geom.P;
    std::vector<double> R1(st.nz, 0.0), R3(st.nz, 0.0);
    for (int z = 0; z < st.nz; ++z)
        for (int r = 0; r < P; ++r) {
            R1[z] += hacc[2 * ((size_t)z * P + r)];
            R3[z] += hacc[2 * ((size_t)z * P + r) + 1];
        }
    const int m = (int)st.knots.size();
    for (int k = 0; k < m; ++k) {
        double g12 = 0.0, g23 = 0.0;
        for (int z = 0; z < st.nz; ++z) {
            const double B = st.basis[(size_t)k * st.nz + z];
            g12 -= B * R1[z];               // x_1 = -d12
            g23 += B * R3[z];               // x_3 = +d23
        }
        grad[k] = g12;
        grad[m + k] = g23;
    }
    if (!std::isfinite(*J)) return fail(st, CTAP_ERR_NONFINITE, "non-finite objective");
    return CTAP_OK;
}

// ------------------------------------------------------------- potentials
template <class T> ctap_status upload_as(PlanState &st, void **d, const std::vector<double> &h)
{
    std::vector<T> c(h.begin(), h.end());
    dev_free(*d);
    return upload(st, d, nullptr, c.data(), c.size() * sizeof(T));
}

ctap_status upload_prec(PlanState &st, void **d, const std::vector<double> &h)
{
    if (st.dtype == CTAP_C64) return upload_as<float>(st, d, h);
    if (st.dtype == CTAP_C128_DF) return upload_as<df>(st, d, h);
    return upload_as<double>(st, d, h);
}

ctap_status upload64(PlanState &st, double **d, const std::vector<double> &h)
{
    void *p = *d;
    dev_free(p);
    *d = nullptr;
    CTAP_TRY(upload(st, &p, nullptr, h.data(), h.size() * sizeof(double)));
    *d = static_cast<double *>(p);
    return CTAP_OK;
}

void clear_potential(PlanState &st)
{
    drop_graphs(st);
    dev_free(st.d_Vd);
    dev_free(st.d_g);
    dev_free(st.d_H);
    dev_free_t(st.d_g64);
    dev_free_t(st.d_H64);
    dev_free_t(st.d_vsep64);
    dev_free(st.d_vz);
    dev_free_t(st.d_vz64);
    st.h_vz.clear();
    st.h_V.clear();
    st.h_vsep.clear();
    st.h_g.clear();
    st.h_H.clear();
    st.vform = VF_NONE;
    st.vmax = 0.0;
    invalidate_sep(st);
}

// max over the grid of |Vx(x) + Vy(y) + Vz(z)|: the sum is extreme where
// every axis term is (the largest or the smallest of each)
double separable_vmax(const PlanState &st)
{
    double hi = 0.0, lo = 0.0;
    size_t o = 0;
    for (int n : {st.nx, st.ny, st.nz}) {
        double mx = st.h_vsep[o], mn = st.h_vsep[o];
        for (int i = 1; i < n; ++i) {
            mx = std::max(mx, st.h_vsep[o + i]);
            mn = std::min(mn, st.h_vsep[o + i]);
        }
        hi += mx;
        lo += mn;
        o += n;
    }
    return std::max(std::fabs(hi), std::fabs(lo));
}

ctap_status set_product(PlanState &st, const std::vector<double> &gy, const std::vector<double> &H)
{
    clear_potential(st);
    st.h_g = gy;
    st.h_H = H;
    double gm = 0.0, hm = 0.0;
    for (double v : gy) gm = std::max(gm, std::fabs(v));
    for (double v : H) hm = std::max(hm, std::fabs(v));
    st.vmax = gm * hm;
    CTAP_TRY(upload_prec(st, &st.d_g, gy));
    CTAP_TRY(upload_prec(st, &st.d_H, H));
    CTAP_TRY(upload64(st, &st.d_g64, gy));
    CTAP_TRY(upload64(st, &st.d_H64, H));
    st.vform = VF_PRODUCT;
    return CTAP_OK;
}

// mid: depth factor of the middle guide per replica (null: 1 for all)
ctap_status set_guides_impl(PlanState &st, double V0, double s, const double *x1z,
                            const double *x3z, double hw, int set_regions,
                            const double *mid = nullptr)
{
    drop_graphs(st);
    if (!(s > 0) || !std::isfinite(V0) || !(hw > 0))
        return fail(st, CTAP_ERR_INVALID_ARG, "guides: need s > 0, finite V0, halfwidth > 0");
    const int nx = st.nx, ny = st.ny, nz = st.nz;
    std::vector<double> gy(ny), H((size_t)nz * nx), D1((size_t)nz * nx), D3((size_t)nz * nx);
    const double inv2s2 = 1.0 / (2.0 * s * s);
    for (int y = 0; y < ny; ++y) {
        const double yy = grid_point(y, ny, st.box[2], st.box[3]);
        gy[y] = std::exp(-yy * yy * inv2s2);
    }
    for (int z = 0; z < nz; ++z) {
        const double c[3] = {x1z[z], 0.0, x3z[z]};
        for (int x = 0; x < nx; ++x) {
            const double xx = grid_point(x, nx, st.box[0], st.box[1]);
            double h = 0.0;
            for (int j = 0; j < 3; ++j) h += std::exp(-(xx - c[j]) * (xx - c[j]) * inv2s2);
            H[(size_t)z * nx + x] = -V0 * h;
            const double d1 = xx - c[0], d3 = xx - c[2];
            D1[(size_t)z * nx + x] = -V0 * std::exp(-d1 * d1 * inv2s2) * d1 / (s * s);
            D3[(size_t)z * nx + x] = -V0 * std::exp(-d3 * d3 * inv2s2) * d3 / (s * s);
        }
    }
    if (st.batch > 1 || mid) {
        // replica b: -V0 (G1 + mid_b G2 + G3); G2 = exp(-x^2/2s^2) (centre 0)
        std::vector<double> Hb((size_t)st.batch * nz * nx);
        for (int b = 0; b < st.batch; ++b) {
            const double m = mid ? mid[b] : 1.0;
            for (int z = 0; z < nz; ++z)
                for (int x = 0; x < nx; ++x) {
                    const double xx = grid_point(x, nx, st.box[0], st.box[1]);
                    const double g2 = std::exp(-xx * xx * inv2s2);
                    Hb[((size_t)b * nz + z) * nx + x] =
                        H[(size_t)z * nx + x] + V0 * (1.0 - m) * g2;
                }
        }
        H.swap(Hb);
    }
    CTAP_TRY(set_product(st, gy, H));
    CTAP_TRY(upload64(st, &st.d_D1, D1));
    CTAP_TRY(upload64(st, &st.d_D3, D3));
    st.have_guides = true;
    st.V0 = V0;
    st.s = s;
    st.h_x1.assign(x1z, x1z + nz);
    st.h_x3.assign(x3z, x3z + nz);
    if (set_regions) {
        st.h_xc.assign((size_t)3 * nz, 0.0);
        for (int z = 0; z < nz; ++z) {
            st.h_xc[z] = x1z[z];
            st.h_xc[(size_t)2 * nz + z] = x3z[z];
        }
        CTAP_TRY(upload64(st, &st.d_xc, st.h_xc));
        st.hw = hw;
        st.have_regions = true;
    }
    return CTAP_OK;
}

bool pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

PlanState *S(ctap_plan_t p) { return p ? &p->st : nullptr; }

}  // namespace

// ====================================================================== ABI
extern "C" {

const char *ctap_version(void) { return "ctap 0.1 (sm_103a)"; }

const char *ctap_status_string(ctap_status s)
{
    switch (s) {
    case CTAP_OK: return "ok";
    case CTAP_ERR_INVALID_ARG: return "invalid argument";
    case CTAP_ERR_UNSUPPORTED_SIZE: return "unsupported grid size";
    case CTAP_ERR_DTYPE: return "dtype mismatch";
    case CTAP_ERR_NO_POTENTIAL: return "no potential set";
    case CTAP_ERR_OOM: return "device allocation failed";
    case CTAP_ERR_CUDA: return "CUDA error";
    case CTAP_ERR_TIMEOUT: return "timeout";
    case CTAP_ERR_NONFINITE: return "non-finite result";
    }
    return "unknown status";
}

const char *ctap_last_error(ctap_plan_t plan)
{
    return plan ? plan->st.err.c_str() : "";
}

ctap_status ctap_plan_create(int nx, int ny, int nz, const double *box, ctap_dtype dtype,
                             void *cuda_stream, ctap_plan_t *out)
{
    return ctap_plan_create_batched(nx, ny, nz, 1, box, dtype, cuda_stream, out);
}

ctap_status ctap_plan_create_batched(int nx, int ny, int nz, int batch, const double *box,
                                     ctap_dtype dtype, void *cuda_stream, ctap_plan_t *out)
{
    if (!out) return CTAP_ERR_INVALID_ARG;
    if (batch < 1 || batch > CTAP_MAX_BATCH) {
        *out = nullptr;
        return CTAP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!box) return CTAP_ERR_INVALID_ARG;
    if (dtype != CTAP_C64 && dtype != CTAP_C128 && dtype != CTAP_C128_DF) return CTAP_ERR_DTYPE;
    for (int i = 0; i < 3; ++i)
        if (!(box[2 * i + 1] > box[2 * i]) || !std::isfinite(box[2 * i]) ||
            !std::isfinite(box[2 * i + 1]))
            return CTAP_ERR_INVALID_ARG;
    if (!pow2(nx) || !pow2(ny) || !pow2(nz) || nx < 8 || ny < 8 || nx > 1024 || ny > 1024 ||
        nz > 1024)
        return CTAP_ERR_UNSUPPORTED_SIZE;
    ctap_plan *p = new (std::nothrow) ctap_plan();
    if (!p) return CTAP_ERR_OOM;
    PlanState &st = p->st;
    st.nx = nx;
    st.ny = ny;
    st.nz = nz;
    std::memcpy(st.box, box, sizeof(st.box));
    st.dtype = dtype;
    st.stream = static_cast<cudaStream_t>(cuda_stream);
    st.esize = dtype == CTAP_C64 ? 8 : 16;
    st.batch = batch;
    st.Nrep = (long long)nx * ny * nz;
    st.N = st.Nrep * batch;
    st.dV = (box[1] - box[0]) / nx * (box[3] - box[2]) / ny * (box[5] - box[4]) / nz;
    const int maxv = dtype == CTAP_C64 ? 32 : 16;
    const int emax = kNT * maxv;
    const char *fg = std::getenv("CTAP_FORCE_GENERIC");
    st.force_generic = fg && fg[0] == '1';
    const char *nr = std::getenv("CTAP_NO_RING");
    st.no_ring = nr && nr[0] == '1';
    const char *npk = std::getenv("CTAP_NO_PACKED");
    st.no_packed = npk && npk[0] == '1';
    try {
        build_geometry(st, emax, maxv);
    } catch (const std::exception &) {
        delete p;
        return CTAP_ERR_UNSUPPORTED_SIZE;
    }
    if (dtype == CTAP_C128_DF) {          // double-float: specialised XY pass for nx = 256,
        st.fast_xy = st.fast_xy && nx == 256;   // specialised Z pass for nz = 1024
        st.fast_z = st.fast_z && nz == 1024;
    }
    auto bail = [&](ctap_status s) {
        ctap_plan_destroy(p);
        return s;
    };
    std::vector<unsigned char> tw;
    build_twiddles(st, tw, maxv);
    ctap_status s = upload(st, &st.d_tw, nullptr, tw.data(), tw.size());
    if (s != CTAP_OK) return bail(s);
    std::vector<double> k2h;
    build_k2h(st, k2h);
    if ((s = upload64(st, &st.d_k2h, k2h)) != CTAP_OK) return bail(s);
    const size_t np = (size_t)5 * xy_grid(st.geom) + z_grid(st.geom) + mask_blocks(st.geom) + 64;
    void *q = nullptr;
    if ((s = dev_alloc(st, &q, np * sizeof(double))) != CTAP_OK) return bail(s);
    st.d_partials = static_cast<double *>(q);
    st.n_partials = np;
    // reductions: 8 doubles per replica, then the imaginary-time scale
    if ((s = dev_alloc(st, &q, (8 * (size_t)batch + 8) * sizeof(double))) != CTAP_OK) return bail(s);
    st.d_red = static_cast<double *>(q);
    st.d_scale = st.d_red + 8 * (size_t)batch;
    *out = p;
    return CTAP_OK;
}

ctap_status ctap_plan_destroy(ctap_plan_t plan)
{
    if (!plan) return CTAP_ERR_INVALID_ARG;
    PlanState &st = plan->st;
    cudaStreamSynchronize(st.stream);
    drop_graphs(st);
    drop_caches(st);
    clear_potential(st);
    dev_free(st.d_tw);
    dev_free(st.d_work);
    dev_free_t(st.d_k2h);
    dev_free_t(st.d_xc);
    dev_free_t(st.d_D1);
    dev_free_t(st.d_D3);
    dev_free_t(st.d_partials);
    dev_free_t(st.d_red);
    dev_free_t(st.d_dens);
    for (auto &e : st.events) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    delete plan;
    return CTAP_OK;
}

ctap_status ctap_set_potential(ctap_plan_t plan, const double *V)
{
    PlanState *st = S(plan);
    if (!st || !V) return CTAP_ERR_INVALID_ARG;
    if (st->batch > 1) return fail(*st, CTAP_ERR_INVALID_ARG, "batched plans take the product form");
    clear_potential(*st);
    st->h_V.assign(V, V + st->N);
    for (double v : st->h_V)
        if (!std::isfinite(v)) return fail(*st, CTAP_ERR_INVALID_ARG, "non-finite potential");
    CTAP_TRY(upload_prec(*st, &st->d_Vd, st->h_V));
    st->vmax = 0.0;
    for (double v : st->h_V) st->vmax = std::max(st->vmax, std::fabs(v));
    st->vform = VF_DENSE;
    st->have_guides = false;
    st->have_spline = false;
    return CTAP_OK;
}

ctap_status ctap_set_potential_wires(ctap_plan_t plan, int nseg, const double *seg,
                                     const double *bias, double mu0_over_4pi, double v_per_field,
                                     double v_offset)
{
    PlanState *st = S(plan);
    if (!st || nseg < 1 || nseg > CTAP_MAX_SEGMENTS || !seg || !bias) return CTAP_ERR_INVALID_ARG;
    if (st->batch > 1) return fail(*st, CTAP_ERR_INVALID_ARG, "batched plans take the product form");
    for (int i = 0; i < 7 * nseg; ++i)
        if (!std::isfinite(seg[i])) return fail(*st, CTAP_ERR_INVALID_ARG, "non-finite segment");
    if (!std::isfinite(bias[0]) || !std::isfinite(bias[1]) || !std::isfinite(bias[2]) ||
        !std::isfinite(mu0_over_4pi) || !std::isfinite(v_per_field) || !std::isfinite(v_offset))
        return fail(*st, CTAP_ERR_INVALID_ARG, "non-finite field parameter");
    void *dseg = nullptr, *dV = nullptr;
    CTAP_TRY(dev_alloc(*st, &dseg, sizeof(double) * 7 * nseg));
    ctap_status rc = dev_alloc(*st, &dV, sizeof(double) * st->N);
    if (rc != CTAP_OK) {
        dev_free(dseg);
        return rc;
    }
    std::vector<double> V(st->N);
    cudaError_t e = cudaMemcpyAsync(dseg, seg, sizeof(double) * 7 * nseg, cudaMemcpyHostToDevice,
                                    st->stream);
    if (e == cudaSuccess) {
        rc = go_other(*st, "wire field", [&] {
            launch_wire_potential(static_cast<double *>(dV), st->geom, static_cast<double *>(dseg),
                                  nseg, bias, mu0_over_4pi, v_per_field, v_offset, st->stream);
        });
        if (rc == CTAP_OK)
            e = cudaMemcpyAsync(V.data(), dV, sizeof(double) * st->N, cudaMemcpyDeviceToHost,
                                st->stream);
    }
    if (e != cudaSuccess) rc = cuda_fail(*st, e, "wire field");
    if (rc == CTAP_OK) rc = wait_stream(*st, 0);
    dev_free(dseg);
    dev_free(dV);
    if (rc != CTAP_OK) return rc;
    return ctap_set_potential(plan, V.data());      // dense form, plan precision
}

ctap_status ctap_set_potential_separable(ctap_plan_t plan, const double *Vx, const double *Vy,
                                         const double *Vz)
{
    PlanState *st = S(plan);
    if (!st || !Vx || !Vy || !Vz) return CTAP_ERR_INVALID_ARG;
    if (st->batch > 1) return fail(*st, CTAP_ERR_INVALID_ARG, "batched plans take the product form");
    clear_potential(*st);
    st->h_vsep.assign(Vx, Vx + st->nx);
    st->h_vsep.insert(st->h_vsep.end(), Vy, Vy + st->ny);
    st->h_vsep.insert(st->h_vsep.end(), Vz, Vz + st->nz);
    for (double v : st->h_vsep)
        if (!std::isfinite(v)) return fail(*st, CTAP_ERR_INVALID_ARG, "non-finite potential");
    CTAP_TRY(upload64(*st, &st->d_vsep64, st->h_vsep));
    st->vform = VF_SEPARABLE;
    st->vmax = separable_vmax(*st);
    st->have_guides = false;
    st->have_spline = false;
    invalidate_sep(*st);
    return CTAP_OK;
}

ctap_status ctap_set_potential_product(ctap_plan_t plan, const double *gy, const double *Hxz)
{
    PlanState *st = S(plan);
    if (!st || !gy || !Hxz) return CTAP_ERR_INVALID_ARG;
    std::vector<double> g(gy, gy + st->ny), H(Hxz, Hxz + (size_t)st->nz * st->nx);
    for (double v : g)
        if (!std::isfinite(v)) return fail(*st, CTAP_ERR_INVALID_ARG, "non-finite potential");
    for (double v : H)
        if (!std::isfinite(v)) return fail(*st, CTAP_ERR_INVALID_ARG, "non-finite potential");
    if (st->batch > 1) {                        // the same H for every replica
        std::vector<double> Hb;
        Hb.reserve(H.size() * st->batch);
        for (int b = 0; b < st->batch; ++b) Hb.insert(Hb.end(), H.begin(), H.end());
        H.swap(Hb);
    }
    CTAP_TRY(set_product(*st, g, H));
    st->have_guides = false;
    st->have_spline = false;
    return CTAP_OK;
}

ctap_status ctap_set_guides(ctap_plan_t plan, double V0, double s, const double *x1z,
                            const double *x3z, double halfwidth, int set_regions)
{
    PlanState *st = S(plan);
    if (!st || !x1z || !x3z) return CTAP_ERR_INVALID_ARG;
    CTAP_TRY(set_guides_impl(*st, V0, s, x1z, x3z, halfwidth, set_regions));
    st->have_spline = false;
    return CTAP_OK;
}

ctap_status ctap_set_guides_batched(ctap_plan_t plan, double V0, double s, const double *x1z,
                                    const double *x3z, const double *mid_scale, double halfwidth,
                                    int set_regions)
{
    PlanState *st = S(plan);
    if (!st || !x1z || !x3z || !mid_scale) return CTAP_ERR_INVALID_ARG;
    for (int b = 0; b < st->batch; ++b)
        if (!std::isfinite(mid_scale[b]))
            return fail(*st, CTAP_ERR_INVALID_ARG, "non-finite middle-guide scale");
    CTAP_TRY(set_guides_impl(*st, V0, s, x1z, x3z, halfwidth, set_regions, mid_scale));
    st->have_spline = false;
    return CTAP_OK;
}

ctap_status ctap_set_guides_spline(ctap_plan_t plan, double V0, double s, int nknots,
                                   const double *knots_z, const double *c12, const double *c23,
                                   double halfwidth, int set_regions)
{
    PlanState *st = S(plan);
    if (!st || !knots_z || !c12 || !c23 || nknots < 2 || nknots > 64) return CTAP_ERR_INVALID_ARG;
    if (st->batch > 1) return fail(*st, CTAP_ERR_INVALID_ARG, "spline controls need an unbatched plan");
    for (int i = 0; i + 1 < nknots; ++i)
        if (!(knots_z[i + 1] > knots_z[i]))
            return fail(*st, CTAP_ERR_INVALID_ARG, "knots must be strictly ascending");
    std::vector<double> knots(knots_z, knots_z + nknots), z(st->nz);
    for (int i = 0; i < st->nz; ++i) z[i] = grid_point(i, st->nz, st->box[4], st->box[5]);
    std::vector<double> B;
    natural_spline_basis(knots, z, B);
    std::vector<double> x1(st->nz, 0.0), x3(st->nz, 0.0);
    for (int m = 0; m < nknots; ++m)
        for (int i = 0; i < st->nz; ++i) {
            x1[i] -= c12[m] * B[(size_t)m * st->nz + i];
            x3[i] += c23[m] * B[(size_t)m * st->nz + i];
        }
    CTAP_TRY(set_guides_impl(*st, V0, s, x1.data(), x3.data(), halfwidth, set_regions));
    st->have_spline = true;
    st->knots = knots;
    st->c12.assign(c12, c12 + nknots);
    st->c23.assign(c23, c23 + nknots);
    st->basis = B;
    return CTAP_OK;
}

ctap_status ctap_add_potential_z(ctap_plan_t plan, const double *Vz)
{
    PlanState *st = S(plan);
    if (!st || !Vz) return CTAP_ERR_INVALID_ARG;
    if (st->vform == VF_NONE) return CTAP_ERR_NO_POTENTIAL;
    const int nx = st->nx, ny = st->ny, nz = st->nz;
    double vzmax = 0.0;
    for (int z = 0; z < nz; ++z) {
        if (!std::isfinite(Vz[z])) return fail(*st, CTAP_ERR_INVALID_ARG, "non-finite potential");
    }
    drop_graphs(*st);
    if (st->vform == VF_DENSE) {
        for (int z = 0; z < nz; ++z)
            for (size_t i = 0; i < (size_t)nx * ny; ++i) st->h_V[(size_t)z * nx * ny + i] += Vz[z];
        CTAP_TRY(upload_prec(*st, &st->d_Vd, st->h_V));
        st->vmax = 0.0;
        for (double v : st->h_V) st->vmax = std::max(st->vmax, std::fabs(v));
    } else if (st->vform == VF_SEPARABLE) {
        for (int z = 0; z < nz; ++z) st->h_vsep[(size_t)nx + ny + z] += Vz[z];
        CTAP_TRY(upload64(*st, &st->d_vsep64, st->h_vsep));
        st->vmax = separable_vmax(*st);
        invalidate_sep(*st);
    } else {
        if (st->h_vz.empty()) st->h_vz.assign(nz, 0.0);
        for (int z = 0; z < nz; ++z) {
            st->h_vz[z] += Vz[z];
            vzmax = std::max(vzmax, std::fabs(st->h_vz[z]));
        }
        CTAP_TRY(upload_prec(*st, &st->d_vz, st->h_vz));
        CTAP_TRY(upload64(*st, &st->d_vz64, st->h_vz));
        double gm = 0.0, hm = 0.0;
        for (double v : st->h_g) gm = std::max(gm, std::fabs(v));
        for (double v : st->h_H) hm = std::max(hm, std::fabs(v));
        st->vmax = gm * hm + vzmax;
    }
    return CTAP_OK;
}

ctap_status ctap_density_xz(ctap_plan_t plan, const void *psi, double *out)
{
    PlanState *st = S(plan);
    if (!st || !psi || !out) return CTAP_ERR_INVALID_ARG;
    const size_t n = (size_t)st->batch * st->nz * st->nx;
    if (!st->d_dens) {
        void *q = nullptr;
        CTAP_TRY(dev_alloc(*st, &q, n * sizeof(double)));
        st->d_dens = static_cast<double *>(q);
    }
    const double dy = (st->box[3] - st->box[2]) / st->ny;
    CTAP_TRY(go_other(*st, "density", [&] {
        if (st->dtype == CTAP_C64)
            launch_density_xz<float>(static_cast<const float2 *>(psi), st->geom, dy, st->d_dens,
                                     st->stream);                    // (complex128 for both others)
        else
            launch_density_xz<double>(static_cast<const double2 *>(psi), st->geom, dy, st->d_dens,
                                      st->stream);
    }));
    cudaError_t e = cudaMemcpyAsync(out, st->d_dens, n * sizeof(double), cudaMemcpyDeviceToHost,
                                    st->stream);
    if (e != cudaSuccess) return cuda_fail(*st, e, "density copy");
    return wait_stream(*st, 0);
}

ctap_status ctap_get_potential(ctap_plan_t plan, double *V)
{
    PlanState *st = S(plan);
    if (!st || !V) return CTAP_ERR_INVALID_ARG;
    if (st->vform == VF_NONE) return CTAP_ERR_NO_POTENTIAL;
    const int nx = st->nx, ny = st->ny, nz = st->nz;
    for (int zb = 0; zb < nz * st->batch; ++zb) {
        const int z = zb % nz;                  // replica-local z
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t i = ((size_t)zb * ny + y) * nx + x;
                double v = 0.0;
                if (st->vform == VF_DENSE) v = st->h_V[i];
                else if (st->vform == VF_SEPARABLE)
                    v = st->h_vsep[x] + st->h_vsep[nx + y] + st->h_vsep[nx + ny + z];
                else v = st->h_g[y] * st->h_H[(size_t)zb * nx + x] +
                         (st->h_vz.empty() ? 0.0 : st->h_vz[z]);
                V[i] = v;
            }
    }
    return CTAP_OK;
}

ctap_status ctap_step(ctap_plan_t plan, void *psi, int nsteps, double dt, ctap_time mode)
{
    PlanState *st = S(plan);
    if (!st || !psi || nsteps < 0 || !std::isfinite(dt)) return CTAP_ERR_INVALID_ARG;
    if (mode != CTAP_REAL && mode != CTAP_IMAG && mode != CTAP_REAL_KVK) return CTAP_ERR_INVALID_ARG;
    if (st->vform == VF_NONE) return CTAP_ERR_NO_POTENTIAL;
    if (reinterpret_cast<uintptr_t>(psi) % st->esize) return fail(*st, CTAP_ERR_INVALID_ARG, "psi misaligned");
    if (mode == CTAP_IMAG && st->batch > 1)
        return fail(*st, CTAP_ERR_INVALID_ARG, "imaginary time needs an unbatched plan");
    if (st->dtype == CTAP_C64)
        return step_maybe_graph<float>(*st, static_cast<float2 *>(psi), nsteps, dt, (int)mode);
    if (st->dtype == CTAP_C128_DF) {
        // complex128 in and out; double-float in between (same 16 bytes per value)
        if (nsteps == 0) return CTAP_OK;
        CTAP_TRY(go_other(*st, "to double-float", [&] { launch_c128_to_df(psi, st->N, st->stream); }));
        CTAP_TRY(step_maybe_graph<df>(*st, static_cast<df2 *>(psi), nsteps, dt, (int)mode));
        return go_other(*st, "from double-float", [&] { launch_df_to_c128(psi, st->N, st->stream); });
    }
    return step_maybe_graph<double>(*st, static_cast<double2 *>(psi), nsteps, dt, (int)mode);
}

ctap_status ctap_observables(ctap_plan_t plan, const void *psi, double *out)
{
    PlanState *st = S(plan);
    if (!st || !psi || !out) return CTAP_ERR_INVALID_ARG;
    std::vector<double> raw(8 * (size_t)st->batch);
    if (st->dtype == CTAP_C64) {
        CTAP_TRY(observe_raw<float>(*st, static_cast<const float2 *>(psi), raw.data()));
    } else if (st->dtype == CTAP_C128_DF) {
        // a double-float copy of the complex128 psi in the work buffer, observed in place
        CTAP_TRY(ensure_work(*st));
        CTAP_TRY(go_other(*st, "to double-float", [&] {
            launch_c128_to_df_copy(psi, st->d_work, st->N, st->stream);
        }));
        CTAP_TRY(observe_raw<df>(*st, static_cast<const df2 *>(st->d_work), raw.data()));
    } else {
        CTAP_TRY(observe_raw<double>(*st, static_cast<const double2 *>(psi), raw.data()));
    }
    for (int b = 0; b < st->batch; ++b)
        CTAP_TRY(finish_observables(*st, raw.data() + 8 * b, out + 6 * b));
    return CTAP_OK;
}

ctap_status ctap_adjoint(ctap_plan_t plan, const void *psi0, int nsteps, double dt, int K,
                         int guide, double *J, double *grad)
{
    PlanState *st = S(plan);
    if (!st || !psi0 || !J || !grad || nsteps < 1 || K < 1 || guide < 1 || guide > 3 ||
        !std::isfinite(dt))
        return CTAP_ERR_INVALID_ARG;
    if (!st->have_spline || !st->have_regions)
        return fail(*st, CTAP_ERR_NO_POTENTIAL, "adjoint needs ctap_set_guides_spline");
    if (st->batch > 1) return fail(*st, CTAP_ERR_INVALID_ARG, "adjoint needs an unbatched plan");
    if (st->dtype == CTAP_C128_DF)
        return fail(*st, CTAP_ERR_DTYPE, "adjoint runs in complex64 or complex128");
    if (st->dtype == CTAP_C64)
        return run_adjoint<float>(*st, static_cast<const float2 *>(psi0), nsteps, dt, K, guide, J,
                                  grad);
    return run_adjoint<double>(*st, static_cast<const double2 *>(psi0), nsteps, dt, K, guide, J,
                               grad);
}

ctap_status ctap_sync(ctap_plan_t plan, int timeout_ms)
{
    PlanState *st = S(plan);
    if (!st) return CTAP_ERR_INVALID_ARG;
    return wait_stream(*st, timeout_ms);
}

ctap_status ctap_set_timeout(ctap_plan_t plan, int timeout_ms)
{
    PlanState *st = S(plan);
    if (!st || timeout_ms <= 0) return CTAP_ERR_INVALID_ARG;
    st->timeout_ms = timeout_ms;
    return CTAP_OK;
}

ctap_status ctap_launch_count(ctap_plan_t plan, long long *count)
{
    PlanState *st = S(plan);
    if (!st || !count) return CTAP_ERR_INVALID_ARG;
    *count = st->launches;
    return CTAP_OK;
}

ctap_status ctap_set_profiling(ctap_plan_t plan, int enable)
{
    PlanState *st = S(plan);
    if (!st) return CTAP_ERR_INVALID_ARG;
    st->profiling = enable != 0;
    return CTAP_OK;
}

ctap_status ctap_pass_times(ctap_plan_t plan, long long counts[3], double ms[3])
{
    PlanState *st = S(plan);
    if (!st || !counts || !ms) return CTAP_ERR_INVALID_ARG;
    CTAP_TRY(wait_stream(*st, 0));
    for (size_t i = 0; i < st->events_used; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, st->events[i].a, st->events[i].b) == cudaSuccess) {
            st->prof_counts[st->events[i].kind] += 1;
            st->prof_ms[st->events[i].kind] += t;
        }
    }
    st->events_used = 0;
    for (int k = 0; k < 3; ++k) {
        counts[k] = st->prof_counts[k];
        ms[k] = st->prof_ms[k];
        st->prof_counts[k] = 0;
        st->prof_ms[k] = 0.0;
    }
    return CTAP_OK;
}

ctap_status ctap_plan_info(ctap_plan_t plan, long long info[5])
{
    PlanState *st = S(plan);
    if (!st || !info) return CTAP_ERR_INVALID_ARG;
    info[0] = st->geom.P;
    info[1] = st->geom.Ly;
    info[2] = st->geom.C;
    info[3] = st->N * st->esize;
    const bool ring = st->fast_z && !st->no_ring && st->dtype == CTAP_C64 && st->nz == 1024 &&
                      st->geom.P == 4 && st->geom.w == 4;
    // the steady XY ring passes take the product form; the packed one also
    // the separable form
    const bool xy_ring_geom = st->fast_xy && !st->no_ring && st->dtype == CTAP_C64 && st->nx == 256 &&
                              st->geom.Ly == 64;
    const bool xy_packed = xy_ring_geom && !st->no_packed && packed_xy_supported(st->geom) &&
                           (st->vform == VF_PRODUCT || st->vform == VF_SEPARABLE);
    const bool xy_ring = xy_ring_geom && (st->vform == VF_PRODUCT || xy_packed);
    info[4] = (st->fast_xy ? 1 : 0) | (st->fast_z ? 2 : 0) | (ring ? 4 : 0) | (xy_ring ? 8 : 0) |
              (packed_z_on(*st) ? 16 : 0) | (xy_packed ? 32 : 0);
    return CTAP_OK;
}

}  // extern "C"
