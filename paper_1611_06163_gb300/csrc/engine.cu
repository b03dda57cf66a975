// Host runtime behind the C ABI of tdpd.h: replica descriptions, device
// layout, membrane topology tables, the captured per-step CUDA graphs, and
// the read-back paths.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "launch.h"

using namespace tdpd;

namespace {

constexpr int GRAPH_LONG = 16;   // steps per long graph (even: keeps the buffer parity)

struct HostRbc {
    int nv = 0, ntri = 0, type = 1;
    std::vector<int32_t> tri;
    std::vector<float> rest;   // nv*3
};

struct HostRep {
    tdpd_config cfg{};
    float a[MAXT * MAXT] = {}, gamma[MAXT * MAXT] = {}, sigma[MAXT * MAXT] = {};
    float kappa[MAXT * MAXT * MAXS] = {};
    float k_react = 0.f;
    int r_src = 0, r_dst = 0;
    uint32_t r_types = 0;
    tdpd_membrane mem{};
    bool has_mem = false;
    std::vector<float> pos, vel, conc;     // load order
    std::vector<int32_t> type, body;       // body: local membrane index or -1
    std::vector<HostRbc> rbcs;
    int n_free = 0;
    int64_t step = 0;
    int nc[3] = {0, 0, 0};
    int m = 2;
    float skin = 0.0f;     // neighbour-list skin of this replica (0: cell mode)
    float qr_ms = 0.0f, qr_rho = 0.0f;   // random flux (Eq. 7-8); m_s = 0: off
    int fbody_flip = 0;                  // double Poiseuille forcing
    float cyl_R = 0.0f;                  // bounce-back cylinder radius (0: none)
};

struct Topo {
    int nv, ntri, ne;
    std::vector<int32_t> tri;
    std::vector<int> ring_off;         // nv+1, relative
    std::vector<RingEntry> ring;
    std::map<std::pair<int, int>, int> edge_id;
    std::vector<std::pair<int, int>> edges;
};

}  // namespace

struct tdpd_sys {
    std::vector<HostRep> reps;
    bool committed = false;
    std::string err;
    cudaStream_t user = nullptr, own = nullptr, cap = nullptr;
    cudaStream_t side = nullptr;                 // membrane branch of a captured step
    cudaEvent_t fork = nullptr, join = nullptr;
    int N = 0, NC = 0, ns = 0, n_rbc = 0, max_nv = 0;
    int lpp = 1;
    int lanes_fixed = 0;   // 0: timed at commit
    int mode_fixed = 0;    // pair mode: 0 chosen at commit, 1 full shell, 2 half shell
    int sort_fixed = 0;    // list-mode sort: 0 chosen at commit, 1 kernel chain, 2 one cluster
    int sort_ctas = 0;     // CTAs of the one-cluster sort in use (0: the kernel chain)
    std::vector<float> sort_ms;    // commit's timing of the two sorts (ms per 16 steps: cluster, chain)
    std::vector<float> shape_ms;   // commit's timing of the candidate list shapes (ms per 16 steps)
    int shape_win = -1;            // the shape chosen (-1: not timed)
    struct {
        float skin;
        int m;
    } shape = {0.0f, 0};           // the list shape in use (m 0: each replica's configured width)
    bool half = false;     // list mode with half-shell lists (each unordered pair once)
    long long *accF = nullptr, *accQ = nullptr;   // half shell: partners' fixed-point shares
    float4 *fown = nullptr;                       // half shell: own force sums
    float *qown = nullptr;                        // half shell: own flux sums
    float skin = -1.0f;    // neighbour-list skin; 0: cell mode; < 0: default
    bool use_list = false;
    int *nl = nullptr, *nlc = nullptr;   // neighbour lists (own allocation: resized by the lane count)
    int nl_cap = 0;
    size_t nl_ints = 0;
    float4 *xb = nullptr;
    uint32_t *disp[2] = {nullptr, nullptr}, *rb = nullptr, *rb_all = nullptr;
    uint32_t *builds = nullptr;          // list rebuild steps per replica (since commit)
    int parity = 0;
    int64_t step = 0;
    Buffers buf[2] = {};
    std::vector<void *> allocs;
    float4 *fext = nullptr, *mx = nullptr, *mv = nullptr;   // load order
    int *inv = nullptr, *count = nullptr, *cell_start = nullptr;
    int *tile_sum[2] = {nullptr, nullptr};
    int n_tiles = 0;
    int4 *d_chunks = nullptr;
    std::vector<int4> h_chunks;
    int2 *cellrank = nullptr, *keys = nullptr;
    uint32_t *errw = nullptr, *step_ctr = nullptr;
    uint32_t *quar = nullptr;            // per replica: quarantined this step (set by the gather)
    RepParams *d_reps = nullptr;
    RbcDev *d_rbcs = nullptr;
    int *d_tri = nullptr;
    FanEntry *d_fan = nullptr;
    float *d_a0j = nullptr;
    float2 *d_bond = nullptr;
    float4 *d_ref[2] = {nullptr, nullptr};
    double2 *d_av[2] = {nullptr, nullptr};   // (A, V) per membrane, written by step parity
    float2 *d_cgv[2] = {nullptr, nullptr};   // their constraint coefficients
    bool all_lagged = false;                 // every membrane's K-Apply uses the previous totals
    cudaEvent_t gathered = nullptr;          // lagged: K-Gather done on the side stream
    double *d_obs = nullptr, *d_obs_tot = nullptr;
    unsigned *d_obs_done = nullptr;
    float *d_in = nullptr;              // uploaded x, v, C of a loaded state (load order)
    int4 *d_wstat = nullptr;            // fixed bits of each particle (load order)
    uint32_t *d_flag = nullptr;         // check result of a state loaded from device memory
    cudaGraphExec_t ginit = nullptr;    // forces of a loaded state
    // pinned host staging of loaded states and observables (async copies);
    // stage_done marks the end of the last copies out of it
    unsigned char *h_stage = nullptr;
    size_t h_stage_bytes = 0;
    double *h_obs = nullptr;
    cudaEvent_t stage_done = nullptr;
    std::vector<int> rep_pbase, rep_rbc0;
    std::vector<RbcDev> h_rbcs;
    std::vector<Topo> topos;
    cudaGraphExec_t g1[2] = {nullptr, nullptr}, glong[2] = {nullptr, nullptr}, gtimed[2] = {nullptr, nullptr};
    cudaEvent_t ev[12] = {};
    int n_ev = 0;
};

namespace {

thread_local std::string g_err;

tdpd_status fail(tdpd_sys *s, tdpd_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    g_err = buf;
    return code;
}

#define CU(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return fail(s, TDPD_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                         \
    } while (0)

cudaStream_t exec_stream(tdpd_sys *s) { return s->user ? s->user : s->own; }

template <class T>
tdpd_status dalloc(tdpd_sys *s, T **p, size_t n)
{
    void *q = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T));
    if (e != cudaSuccess) return fail(s, TDPD_ENOMEM, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
    s->allocs.push_back(q);
    *p = (T *)q;
    return TDPD_OK;
}

template <class T>
tdpd_status upload(tdpd_sys *s, T *dst, const T *src, size_t n)
{
    if (n == 0) return TDPD_OK;
    CU(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, exec_stream(s)));
    return TDPD_OK;
}

double min_image_d(double d, double L, int periodic)
{
    if (!periodic) return d;
    return d - L * std::floor(d / L + 0.5);
}

// Build the one-ring tables of a closed oriented triangulation.
tdpd_status build_topo(tdpd_sys *s, int nv, int ntri, const int32_t *tri, Topo &T)
{
    T.nv = nv;
    T.ntri = ntri;
    T.tri.assign(tri, tri + 3 * ntri);
    std::map<std::pair<int, int>, int> opp;   // directed edge -> third vertex
    std::map<std::pair<int, int>, int> dtri;  // directed edge -> triangle
    for (int t = 0; t < ntri; ++t) {
        for (int k = 0; k < 3; ++k) {
            int a = tri[3 * t + k], b = tri[3 * t + (k + 1) % 3], c = tri[3 * t + (k + 2) % 3];
            if (a < 0 || a >= nv || a == b || b == c || a == c)
                return fail(s, TDPD_EINVAL, "triangle %d has a bad vertex index", t);
            auto key = std::make_pair(a, b);
            if (opp.count(key)) return fail(s, TDPD_EINVAL, "directed edge (%d,%d) occurs twice: mesh not consistently oriented", a, b);
            opp[key] = c;
            dtri[key] = t;
        }
    }
    for (auto &kv : opp) {
        auto rev = std::make_pair(kv.first.second, kv.first.first);
        if (!opp.count(rev)) return fail(s, TDPD_EINVAL, "edge (%d,%d) has one triangle: mesh not closed", kv.first.first, kv.first.second);
        if (kv.first.first < kv.first.second) {
            T.edge_id[kv.first] = (int)T.edges.size();
            T.edges.push_back(kv.first);
        }
    }
    T.ne = (int)T.edges.size();
    if (nv - T.ne + ntri != 2) return fail(s, TDPD_EINVAL, "V - E + F = %d, not a closed genus-0 surface", nv - T.ne + ntri);
    auto eid = [&](int a, int b) { return T.edge_id[std::make_pair(std::min(a, b), std::max(a, b))]; };
    // fan of each vertex: triangles (v, a, b) chain a -> b
    std::vector<std::vector<std::pair<int, int>>> fan(nv);   // (a, triangle) keyed by a, next b
    std::vector<std::map<int, int>> next(nv), ftri(nv);
    for (int t = 0; t < ntri; ++t)
        for (int k = 0; k < 3; ++k) {
            int v = tri[3 * t + k], a = tri[3 * t + (k + 1) % 3], b = tri[3 * t + (k + 2) % 3];
            next[v][a] = b;
            ftri[v][a] = t;
        }
    T.ring_off.assign(nv + 1, 0);
    for (int v = 0; v < nv; ++v) {
        int deg = (int)next[v].size();
        if (deg < 3) return fail(s, TDPD_EINVAL, "vertex %d has degree %d", v, deg);
        T.ring_off[v] = (int)T.ring.size();
        int a0 = next[v].begin()->first, a = a0;
        for (int l = 0; l < deg; ++l) {
            auto it = next[v].find(a);
            if (it == next[v].end()) return fail(s, TDPD_EINVAL, "vertex %d: open fan", v);
            int b = it->second;
            RingEntry E;
            E.nb = a;
            E.edge = eid(v, a);
            E.tri = ftri[v][a];
            E.across = opp[std::make_pair(b, a)];
            T.ring.push_back(E);
            a = b;
        }
        if (a != a0) return fail(s, TDPD_EINVAL, "vertex %d: fan is not a single cycle", v);
    }
    T.ring_off[nv] = (int)T.ring.size();
    return TDPD_OK;
}

// Unwrap a membrane (nv*3 floats) by walking edges with the minimum image.
void unwrap(const HostRep &R, const Topo &T, const float *p, std::vector<double> &x)
{
    const int nv = T.nv;
    x.assign(3 * (size_t)nv, 0.0);
    std::vector<char> done(nv, 0);
    std::vector<int> stack{0};
    for (int c = 0; c < 3; ++c) x[c] = p[c];
    done[0] = 1;
    while (!stack.empty()) {
        int v = stack.back();
        stack.pop_back();
        for (int k = T.ring_off[v]; k < T.ring_off[v + 1]; ++k) {
            int u = T.ring[k].nb;
            if (done[u]) continue;
            for (int c = 0; c < 3; ++c)
                x[3 * u + c] = x[3 * v + c] + min_image_d((double)p[3 * u + c] - p[3 * v + c], R.cfg.L[c], R.cfg.periodic[c]);
            done[u] = 1;
            stack.push_back(u);
        }
    }
}

RepParams make_params(const HostRep &R, int cell_base, int pbase, int n)
{
    RepParams P;
    std::memset(&P, 0, sizeof P);
    const tdpd_config &c = R.cfg;
    for (int k = 0; k < 3; ++k) {
        P.L[k] = c.L[k];
        P.nc[k] = R.nc[k];
        P.cell_scale[k] = (float)((double)R.nc[k] / (double)c.L[k]);
        P.h[k] = (float)((double)c.L[k] / (double)R.nc[k]);
        P.periodic[k] = c.periodic[k];
        P.fbody[k] = c.body_force[k];
    }
    P.cell_base = cell_base;
    P.n_cells = R.nc[0] * R.nc[1] * R.nc[2];
    P.m_stencil = R.m;
    P.pbase = pbase;
    P.n = n;
    P.wall_lo = c.wall_lo;
    P.wall_hi = c.wall_hi;
    P.seed_lo = (uint32_t)(c.seed & 0xffffffffu);
    P.seed_hi = (uint32_t)(c.seed >> 32);
    P.step0 = (uint32_t)R.step;
    P.ntypes = c.n_types;
    P.ns = c.n_species;
    P.dt = c.dt;
    P.hdt = (float)(0.5 * c.dt);
    P.hdt2 = (float)(0.5 * (double)c.dt * c.dt);
    P.ldt = (float)((double)c.lambda * c.dt);
    P.inv_sqrt_dt = (float)(1.0 / std::sqrt((double)c.dt));
    P.rc2 = c.rc * c.rc;
    P.inv_rc = (float)(1.0 / c.rc);
    P.rcc2 = c.rcc * c.rcc;
    P.inv_rcc = c.rcc > 0 ? (float)(1.0 / c.rcc) : 0.f;
    const float rcut = std::max(c.rc, c.rcc);
    P.rcut2 = rcut * rcut;
    P.rlist2 = (rcut + R.skin) * (rcut + R.skin);
    P.half_skin2 = 0.25f * R.skin * R.skin;
    for (int k = 0; k < 3; ++k) P.inv_L[k] = c.periodic[k] ? (float)(1.0 / (double)c.L[k]) : 0.0f;
    P.sR = 0.5f * c.s_f;
    P.s_c = c.s_c;
    P.sR_is1 = (P.sR == 1.0f);
    P.sc_is2 = (c.s_c == 2.0f);
    std::memcpy(P.a, R.a, sizeof P.a);
    std::memcpy(P.gamma, R.gamma, sizeof P.gamma);
    std::memcpy(P.sigma, R.sigma, sizeof P.sigma);
    // kappa packed as [ti*T + tj][ns] for the replica's own T and ns
    const int T = c.n_types, S = c.n_species;
    for (int i = 0; i < T; ++i)
        for (int j = 0; j < T; ++j)
            for (int k = 0; k < S; ++k) P.kappa[(i * T + j) * S + k] = R.kappa[(i * MAXT + j) * MAXS + k];
    for (int i = 0; i < T; ++i)
        for (int j = 0; j < T; ++j) {
            P.a[i * T + j] = R.a[i * MAXT + j];
            P.gamma[i * T + j] = R.gamma[i * MAXT + j];
            P.sigma[i * T + j] = R.sigma[i * MAXT + j];
        }
    P.frozen_mask = c.frozen_types;
    P.react_mask = R.r_types;
    P.k_react = R.k_react;
    P.r_src = R.r_src;
    P.r_dst = R.r_dst;
    P.exclude_same_body = c.exclude_same_body;
    const tdpd_membrane &m = R.mem;
    P.m_kT = m.kT; P.m_p = m.p; P.m_x0 = m.x0; P.m_m = m.m;
    P.m_kg = m.kg; P.m_kl = m.kl; P.m_kv = m.kv; P.m_kb = m.kb;
    P.m_cos0 = (float)std::cos((double)m.theta0);
    P.m_sin0 = (float)std::sin((double)m.theta0);
    P.m_gT = m.gammaT; P.m_gC = m.gammaC;
    P.m_wlc0 = m.p > 0 ? (float)((double)m.kT / m.p) : 0.f;
    const double s0 = std::sqrt(2.0 * (double)m.kT / c.dt);
    P.m_rand_T = (float)(s0 * std::sqrt(2.0 * (double)m.gammaT));
    P.m_rand_C = (float)(s0 * std::sqrt(std::max(0.0, 3.0 * (double)m.gammaC - m.gammaT)) / 3.0);
    P.m_lagged = m.lagged_av != 0;
    P.qr_coef = R.qr_ms > 0.0f ? (float)((double)R.qr_ms * std::sqrt((double)R.qr_rho)) : 0.0f;
    P.fbody_flip = R.fbody_flip;
    P.cyl_R = R.cyl_R;
    P.cyl_c[0] = 0.5f * R.cfg.L[1];
    P.cyl_c[1] = 0.5f * R.cfg.L[2];
    return P;
}

}  // namespace

RepParams tdpd::build_rep_params(const tdpd_config &c, const float *pair_coef, const float *kappa,
                                 const int nc[3], int m, int cell_base, int pbase, int n)
{
    HostRep R;
    R.cfg = c;
    const int T = c.n_types, S = c.n_species;
    for (int i = 0; i < T; ++i)
        for (int j = 0; j < T; ++j) {
            R.a[i * MAXT + j] = pair_coef[(i * T + j) * 3];
            R.gamma[i * MAXT + j] = pair_coef[(i * T + j) * 3 + 1];
            R.sigma[i * MAXT + j] = pair_coef[(i * T + j) * 3 + 2];
            for (int k = 0; k < S; ++k) R.kappa[(i * MAXT + j) * MAXS + k] = kappa[(i * T + j) * S + k];
        }
    for (int k = 0; k < 3; ++k) R.nc[k] = nc[k];
    R.m = m;
    return make_params(R, cell_base, pbase, n);
}

void tdpd::set_thread_error(const char *msg) { g_err = msg; }

bool tdpd::config_error(const tdpd_config &c, char *msg, size_t len)
{
    auto why = [&](const char *fmt, int v = 0) {
        std::snprintf(msg, len, fmt, v);
        return true;
    };
    for (int k = 0; k < 3; ++k)
        if (!(c.L[k] > 0) || !std::isfinite(c.L[k])) return why("box edge %d must be positive and finite", k);
    if (!c.periodic[0] || !c.periodic[1]) return why("x and y must be periodic (walls only along z)");
    if (!c.periodic[2] && !(c.wall_lo >= 0 && c.wall_lo < c.wall_hi && c.wall_hi <= c.L[2]))
        return why("walls need 0 <= wall_lo < wall_hi <= L[2]");
    if (c.n_types < 1 || c.n_types > MAXT) return why("n_types must be in 1..%d", MAXT);
    if (c.n_species < 1 || c.n_species > MAXS) return why("n_species must be in 1..%d", MAXS);
    if (!(c.dt > 0) || !std::isfinite(c.dt)) return why("dt must be positive and finite");
    if (!(c.rc > 0) || !(c.rcc >= 0) || !std::isfinite(c.rc) || !std::isfinite(c.rcc))
        return why("cut-offs: rc > 0, rcc >= 0, both finite");
    if (!(c.s_f > 0) || !(c.s_c > 0)) return why("weight exponents must be positive");
    if (c.frozen_types >> c.n_types) return why("frozen_types names a type >= n_types (%d)", c.n_types);
    if (c.cells_per_cutoff < 0 || c.cells_per_cutoff > 3) return why("cells_per_cutoff must be 0, 1, 2 or 3");
    return false;
}

namespace {

tdpd_status free_device(tdpd_sys *s)
{
    for (int p = 0; p < 2; ++p) {
        if (s->g1[p]) cudaGraphExecDestroy(s->g1[p]);
        if (s->glong[p]) cudaGraphExecDestroy(s->glong[p]);
        if (s->gtimed[p]) cudaGraphExecDestroy(s->gtimed[p]);
        s->g1[p] = s->glong[p] = s->gtimed[p] = nullptr;
    }
    if (s->ginit) cudaGraphExecDestroy(s->ginit);
    s->ginit = nullptr;
    for (int k = 0; k < s->n_ev; ++k) cudaEventDestroy(s->ev[k]);
    s->n_ev = 0;
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->join) cudaEventDestroy(s->join);
    if (s->gathered) cudaEventDestroy(s->gathered);
    s->gathered = nullptr;
    if (s->side) cudaStreamDestroy(s->side);
    s->fork = s->join = nullptr;
    s->side = nullptr;
    for (void *p : s->allocs) cudaFree(p);
    s->allocs.clear();
    if (s->nl) cudaFree(s->nl);
    s->nl = nullptr;
    s->nl_ints = 0;
    s->nl_cap = 0;
    if (s->stage_done) cudaEventSynchronize(s->stage_done), cudaEventDestroy(s->stage_done);
    if (s->h_stage) cudaFreeHost(s->h_stage);
    s->stage_done = nullptr;
    s->h_stage = nullptr;
    s->h_obs = nullptr;
    s->h_stage_bytes = 0;
    return TDPD_OK;
}

const char *const KERNEL_NAMES[] = {"scan",       "scatter_keys", "rank_gather", "mem_gather", "mem_forces",
                                    "pair",       "decide",       "bin",         "list_build", "sort"};

// ref_in: which reference point buffer this evaluation reads; its K-Gather
// writes the other one and the (A, V) buffer of the same index. inc: a step
// (advance the membrane step counter); the forces of a loaded state (inc 0)
// use their own totals even where the constraints are lagged.
MemArgs mem_args(tdpd_sys *s, int ref_in, int inc)
{
    const int q = 1 - ref_in;
    MemArgs m{};
    m.mx = s->mx; m.mv = s->mv; m.reps = s->d_reps; m.rbcs = s->d_rbcs;
    m.tri = s->d_tri; m.fan = s->d_fan;
    m.a0j = s->d_a0j; m.bond = s->d_bond; m.ref_in = s->d_ref[ref_in]; m.ref_out = s->d_ref[1 - ref_in];
    m.av_out = s->d_av[q]; m.cgv_out = s->d_cgv[q]; m.cgv_seq = s->d_cgv[q];
    m.cgv_lag = inc ? s->d_cgv[1 - q] : s->d_cgv[q];
    m.fext = s->fext; m.n_rbc = s->n_rbc; m.max_nv = s->max_nv;
    m.mem_ctr = s->step_ctr + 1; m.q = q;
    return m;
}

// disp_next: where list mode records the displacements of the next positions
// build_rb (list mode): the replicas whose lanes build their lists inside
// the pair kernel first (a rebuild step)
PairArgs pair_args(tdpd_sys *s, const Buffers &b, int integrate, int *tile_sum, uint32_t *disp_next = nullptr,
                   const uint32_t *build_rb = nullptr)
{
    PairArgs a{};
    a.tile_sum = tile_sum;
    a.b = b; a.fext = s->fext; a.mx = s->mx; a.mv = s->mv; a.reps = s->d_reps; a.cell_start = s->cell_start; a.count = s->count;
    a.cellrank = s->cellrank; a.err = s->errw; a.quar = s->quar; a.step_ctr = s->step_ctr; a.n = s->N; a.ns = s->ns;
    a.integrate = integrate;
    a.lpp = s->lpp;
    a.std_exp = 1;
    for (const HostRep &R : s->reps) {
        if (R.qr_ms > 0.0f) a.qr = 1;
        if (!(R.cfg.s_f == 2.0f && R.cfg.s_c == 2.0f)) a.std_exp = 0;
    }
    if (s->use_list) {
        a.pre = b.pos == s->buf[0].pos ? s->buf[1] : s->buf[0];
        a.nl = s->nl; a.nlc = s->nlc; a.cap = s->nl_cap; a.xb = s->xb; a.disp_next = disp_next;
        a.half = s->half ? 1 : 0;
        a.accF = s->accF; a.accQ = s->accQ; a.fown = s->fown; a.qown = s->qown;
        if (build_rb) {
            a.rb = build_rb;
            a.nl_w = s->nl; a.nlc_w = s->nlc; a.xb_w = s->xb;
            a.m2 = 1;
            for (const HostRep &R : s->reps) a.m2 = a.m2 && R.m == 2;
        }
    }
    return a;
}

// List build over the sorted buffer b for the replicas flagged in rb.
ListArgs list_args(tdpd_sys *s, const Buffers &b, const uint32_t *rb, int cap)
{
    ListArgs l{};
    l.pos = b.pos; l.vel = b.vel; l.reps = s->d_reps; l.cell_start = s->cell_start; l.rb = rb; l.quar = s->quar;
    l.n_rep = (int)s->reps.size();
    l.nl = s->nl; l.nlc = s->nlc; l.xb = s->xb; l.err = s->errw; l.n = s->N; l.lpp = s->lpp; l.cap = cap;
    l.m2 = 1;
    for (const HostRep &R : s->reps) l.m2 = l.m2 && R.m == 2;
    l.half = s->half ? 1 : 0;
    return l;
}

// The gather of each step derives the quarantine from the status words.
Quarantine quarantine(tdpd_sys *s)
{
    Quarantine q;
    q.err = s->errw;
    q.quar = s->quar;
    q.n_reps = (int)s->reps.size();
    return q;
}

// Up to this many replicas every binning CTA takes the rebuild decision
// itself (it reads each replica's maximum), saving the one-CTA decision
// kernel's launch; more replicas keep the separate kernel.
constexpr int DECIDE_INLINE_MAX = 16;
bool inline_decide(const tdpd_sys *s) { return (int)s->reps.size() <= DECIDE_INLINE_MAX; }

// List mode with one or two species (and no random flux): the pair kernel
// (its one- and two-species forms) builds the lists of rebuilding replicas
// itself; otherwise k_list_build runs before it.
bool pair_builds_lists(const tdpd_sys *s)
{
    if (!s->use_list || s->ns > 2) return false;
    for (const HostRep &R : s->reps)
        if (R.qr_ms > 0.0f) return false;
    return true;
}

// The one-cluster sort of step p (reading buffer p): its decision reads the
// maxima of the last epilogue, like k_bin_next's inline decision.
SortSmallArgs sort_small_args(tdpd_sys *s, int p)
{
    SortSmallArgs a;
    a.cur = s->buf[p];
    a.nxt = s->buf[1 - p];
    a.reps = s->d_reps;
    a.n = s->N;
    a.ns_rt = s->ns;
    a.nc = s->NC;
    a.count = s->count;
    a.cell_start = s->cell_start;
    a.inv = s->inv;
    a.cellrank = s->cellrank;
    a.keys = s->keys;
    a.D = DecideArgs{s->disp[p], s->disp[1 - p], s->rb, s->step_ctr, s->builds, (int)s->reps.size()};
    a.Qa = quarantine(s);
    return a;
}

// Cells the one-cluster sort may scan (its particle limit depends on the
// cluster size: SORT_SMALL_ITEMS per thread).
constexpr int SORT_SMALL_MAX_NC = 1 << 20;

// Kernel kinds one step launches, in order (indices into KERNEL_NAMES).
std::vector<int> step_kernels(const tdpd_sys *s)
{
    std::vector<int> k;
    if (s->use_list) {
        if (s->sort_ctas) k = {9};
        else if (inline_decide(s)) k = {7, 0, 1, 2};
        else k = {6, 7, 0, 1, 2};
        if (!pair_builds_lists(s)) k.push_back(8);
    } else {
        k = {0, 1, 2};
    }
    if (s->n_rbc) { k.push_back(3); k.push_back(4); }
    k.push_back(5);
    return k;
}

// Enqueue one step reading buffer p and leaving the state in buffer 1-p. With
// ev (one event per kernel plus one), event-record nodes bracket each kernel.
void enqueue_step(tdpd_sys *s, int p, cudaStream_t st, cudaEvent_t *ev = nullptr)
{
    const Buffers &cur = s->buf[p], &nxt = s->buf[1 - p];
    int e = 0;
    auto mark = [&]() {
        if (ev && e < s->n_ev) cudaEventRecordWithFlags(ev[e++], st, cudaEventRecordExternal);
    };
    // The membrane kernels read the predicted vertices the last pair epilogue
    // wrote in load order, so they need not wait for the sort: in a plain
    // step they run on a side stream from the step's start. Their forces are
    // needed only by the epilogue, which also writes the vertices' next
    // positions they read, so the branch joins just before the epilogue:
    // before k_pair_finish with the half shell (the branch then overlaps the
    // sort and the pair walk), before the pair kernel otherwise. When every
    // membrane's constraints are lagged, K-Apply goes first and K-Gather (for
    // the next step) follows it on the branch. The timed step keeps one
    // stream, so that the events bracket one kernel each.
    const bool branch = s->n_rbc && !ev;
    if (branch) {
        cudaEventRecord(s->fork, st);
        cudaStreamWaitEvent(s->side, s->fork, 0);
        const MemArgs m = mem_args(s, 1 - p, 1);
        if (s->all_lagged) {
            launch_mem_forces(m, s->side);
            cudaEventRecord(s->join, s->side);
            launch_mem_gather(m, s->side, true);
            cudaEventRecord(s->gathered, s->side);
        } else {
            launch_mem_gather(m, s->side, false);
            launch_mem_forces(m, s->side);
            cudaEventRecord(s->join, s->side);
        }
    }
    mark();
    const int nrep = (int)s->reps.size();
    if (s->use_list) {
        // rebuild the lists of the replicas whose particles moved more than
        // half their skin; the others keep their lists and their slots
        const uint32_t *any = s->rb + nrep;
        if (s->sort_ctas) {
            launch_sort_small(sort_small_args(s, p), s->sort_ctas, st);
            mark();
        } else if (inline_decide(s)) {
            const DecideArgs d{s->disp[p], s->disp[1 - p], s->rb, s->step_ctr, s->builds, nrep};
            launch_bin_next(cur, s->d_reps, s->N, s->count, s->tile_sum[0], s->cellrank, s->rb, any, st, d);
            mark();
        } else {
            launch_rebuild_decide(s->disp[p], s->disp[1 - p], s->rb, s->d_reps, nrep, 0, s->step_ctr, s->builds, st);
            mark();
            launch_bin_next(cur, s->d_reps, s->N, s->count, s->tile_sum[0], s->cellrank, s->rb, any, st);
            mark();
        }
        if (!s->sort_ctas) {
            launch_scan(s->count, s->cell_start, s->n_tiles, s->tile_sum[0], s->tile_sum[1], s->step_ctr, 0, st,
                        any);
            mark();
            launch_scatter_keys(cur, s->cellrank, s->cell_start, s->keys, s->N, st, any, s->rb);
            mark();
            launch_rank_gather(cur, nxt, s->d_reps, s->keys, s->cellrank, s->cell_start, s->inv, s->N, s->ns, 1, st,
                               s->rb, nrep, s->tile_sum[0], s->n_tiles, quarantine(s));
            mark();
        }
        if (!pair_builds_lists(s)) {
            launch_list_build(list_args(s, nxt, s->rb, s->nl_cap), st);
            mark();
        }
    } else {
        launch_scan(s->count, s->cell_start, s->n_tiles, s->tile_sum[p], s->tile_sum[1 - p], s->step_ctr, 1, st);
        mark();
        launch_scatter_keys(cur, s->cellrank, s->cell_start, s->keys, s->N, st);
        mark();
        launch_rank_gather(cur, nxt, s->d_reps, s->keys, s->cellrank, s->cell_start, s->inv, s->N, s->ns, 1, st,
                           nullptr, 0, nullptr, 0, quarantine(s));
        mark();
    }
    if (s->n_rbc && ev) {
        const MemArgs m = mem_args(s, 1 - p, 1);
        launch_mem_gather(m, st, true);
        mark();
        launch_mem_forces(m, st);
        mark();
    }
    const PairArgs pa = pair_args(s, nxt, 1, s->tile_sum[1 - p], s->disp[1 - p],
                                  pair_builds_lists(s) ? s->rb : nullptr);
    auto join = [&]() {
        if (!branch) return;
        cudaStreamWaitEvent(st, s->join, 0);
        if (s->all_lagged) cudaStreamWaitEvent(st, s->gathered, 0);
    };
    if (!s->half) join();
    launch_pair(pa, st, PAIR_WALK);
    if (s->half) join();
    launch_pair(pa, st, PAIR_FINISH);
    mark();
}

constexpr size_t OBS_STAGE = (sizeof(double) * OBS_K + 15) / 16 * 16;
constexpr float DEFAULT_SKIN = 0.2f;   // neighbour-list skin (length units)

// Pinned staging area: observables, the step counters, then x[3N], v[3N],
// C[N*ns] in load order.
uint32_t *stage_ctr(tdpd_sys *s) { return reinterpret_cast<uint32_t *>(s->h_stage + OBS_STAGE); }
float *stage_in(tdpd_sys *s) { return reinterpret_cast<float *>(s->h_stage + OBS_STAGE + 16); }
size_t stage_bytes(int N, int ns)
{
    return OBS_STAGE + 16 + sizeof(float) * (size_t)N * (6 + ns);
}


// fn(lo, hi) over [0, n) in contiguous chunks on up to 16 host threads, one
// thread when n is below min_chunk (the load paths' checks and reference
// points, which would otherwise hold up a large batch's upload)
template <class F>
void host_parallel(size_t n, size_t min_chunk, F fn)
{
    const size_t hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nt = std::min<size_t>({(size_t)16, hw, std::max<size_t>(1, n / std::max<size_t>(1, min_chunk))});
    if (nt <= 1) {
        fn((size_t)0, n);
        return;
    }
    const size_t chunk = (n + nt - 1) / nt;
    std::vector<std::thread> th;
    for (size_t t = 1; t < nt; ++t) {
        const size_t lo = std::min(n, t * chunk), hi = std::min(n, lo + chunk);
        if (lo < hi) th.emplace_back(fn, lo, hi);
    }
    fn((size_t)0, std::min(n, chunk));
    for (std::thread &x : th) x.join();
}

// Batches up to this many particles are checked on the host on load (while
// their upload runs), larger ones on the device.
constexpr int HOST_CHECK_MAX = 1 << 17;

// First particle (load index over the whole batch) of pos/vel outside its
// replica's box or with a non-finite velocity, or -1; contiguous chunks of
// the batch are checked in parallel.
long first_bad_particle(const tdpd_sys *s, const float *pos, const float *vel)
{
    std::mutex m;
    long first = -1;
    host_parallel((size_t)s->N, (size_t)1 << 16, [&](size_t lo, size_t hi) {
        // the replicas overlapping [lo, hi), each with its box in registers
        size_t r = (size_t)(std::upper_bound(s->rep_pbase.begin(), s->rep_pbase.end(), (int)lo) -
                            s->rep_pbase.begin()) - 1;
        for (size_t i0 = lo; i0 < hi; ++r) {
            const size_t end = std::min(hi, r + 1 < s->reps.size() ? (size_t)s->rep_pbase[r + 1] : hi);
            const float L0 = s->reps[r].cfg.L[0], L1 = s->reps[r].cfg.L[1], L2 = s->reps[r].cfg.L[2];
            for (size_t i = i0; i < end; ++i) {
                const float *x = pos + 3 * i, *v = vel + 3 * i;
                const bool ok = x[0] >= 0.0f && x[0] < L0 && x[1] >= 0.0f && x[1] < L1 && x[2] >= 0.0f &&
                                x[2] < L2 && std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
                if (!ok) {
                    std::lock_guard<std::mutex> g(m);
                    if (first < 0 || (long)i < first) first = (long)i;
                    return;
                }
            }
            i0 = end;
        }
    });
    return first;
}



// Forces of a freshly loaded state: pack the uploaded load-order arrays into
// buffer 0 (F = Q = 0), bin and sort into buffer 1, pair forces there (no
// integration). The membrane kernels read the packed vertices in load order,
// so outside the timed set-up they run on the side stream beside the sort.
void enqueue_init(tdpd_sys *s, cudaStream_t st, bool branch)
{
    const int N = s->N, ns = s->ns;
    cudaMemsetAsync(s->count, 0, sizeof(int) * (size_t)s->n_tiles * SCAN_TILE, st);
    cudaMemsetAsync(s->tile_sum[0], 0, sizeof(int) * s->n_tiles, st);
    cudaMemsetAsync(s->tile_sum[1], 0, sizeof(int) * s->n_tiles, st);
    cudaMemsetAsync(s->errw, 0, sizeof(uint32_t) * s->reps.size(), st);
    cudaMemsetAsync(s->quar, 0, sizeof(uint32_t) * s->reps.size(), st);
    cudaMemsetAsync(s->fext, 0, sizeof(float4) * N, st);
    launch_pack_state(s->d_in, s->d_wstat, s->buf[0], s->mx, s->mv, N, ns, st);
    branch = branch && s->n_rbc;
    if (branch) {
        cudaEventRecord(s->fork, st);
        cudaStreamWaitEvent(s->side, s->fork, 0);
        const MemArgs m = mem_args(s, 1, 0);
        launch_mem_gather(m, s->side, false);
        launch_mem_forces(m, s->side);
        cudaEventRecord(s->join, s->side);
    }
    launch_bin_init(s->buf[0], s->d_reps, N, s->count, s->tile_sum[0], s->cellrank, st);
    launch_scan(s->count, s->cell_start, s->n_tiles, s->tile_sum[0], s->tile_sum[1], s->step_ctr, 0, st);
    launch_scatter_keys(s->buf[0], s->cellrank, s->cell_start, s->keys, N, st);
    if (s->use_list) {
        launch_rank_gather(s->buf[0], s->buf[1], s->d_reps, s->keys, s->cellrank, s->cell_start, s->inv, N, ns, 0,
                           st, nullptr, 0, s->tile_sum[0], s->n_tiles, quarantine(s));
        cudaMemsetAsync(s->disp[1], 0, sizeof(uint32_t) * s->reps.size(), st);
        // (the one- and two-species pair kernels build every lane's list
        // themselves, as on a step where every replica rebuilds)
        if (!pair_builds_lists(s)) launch_list_build(list_args(s, s->buf[1], s->rb_all, s->nl_cap), st);
    } else {
        launch_rank_gather(s->buf[0], s->buf[1], s->d_reps, s->keys, s->cellrank, s->cell_start, s->inv, N, ns, 0,
                           st, nullptr, 0, nullptr, 0, quarantine(s));
    }
    if (s->n_rbc && !branch) {
        const MemArgs m = mem_args(s, 1, 0);
        launch_mem_gather(m, st, true);
        launch_mem_forces(m, st);
    }
    const PairArgs pa = pair_args(s, s->buf[1], 0, s->tile_sum[1], s->disp[1],
                                  s->use_list && pair_builds_lists(s) ? s->rb_all : nullptr);
    if (branch && !s->half) cudaStreamWaitEvent(st, s->join, 0);
    launch_pair(pa, st, PAIR_WALK);
    if (branch && s->half) cudaStreamWaitEvent(st, s->join, 0);
    launch_pair(pa, st, PAIR_FINISH);
}

// Device part of loading a state whose load-order arrays are staged
// (upload_in) or already in d_in: the membranes' reference points, then the
// forces of the state.
tdpd_status init_device(tdpd_sys *s, bool upload_in)
{
    cudaStream_t st = exec_stream(s);
    tdpd_status rc;
    if (upload_in && (rc = upload(s, s->d_in, stage_in(s), (size_t)s->N * (6 + s->ns)))) return rc;
    int max_stride = 0;
    for (const RbcDev &D : s->h_rbcs) max_stride = std::max(max_stride, D.fan_stride);
    launch_mem_ref(s->d_in, s->d_rbcs, s->d_fan, s->d_reps, s->d_ref[1], s->n_rbc, s->max_nv, max_stride, st);
    uint32_t *ctr = stage_ctr(s);
    ctr[0] = ctr[1] = ctr[2] = (uint32_t)s->step;        // sort / pair, membrane (by parity)
    if ((rc = upload(s, s->step_ctr, ctr, 3))) return rc;
    CU(cudaEventRecord(s->stage_done, st));
    if (s->ginit) CU(cudaGraphLaunch(s->ginit, st));
    else enqueue_init(s, st, false);
    CU(cudaGetLastError());
    s->parity = 1;
    return TDPD_OK;
}

// Load every replica's host state (load order) and compute its forces.
tdpd_status init_state(tdpd_sys *s)
{
    const int N = s->N, ns = s->ns;
    CU(cudaEventSynchronize(s->stage_done));          // the pinned area is free
    float *x3 = stage_in(s), *v3 = x3 + 3 * (size_t)N, *c = v3 + 3 * (size_t)N;
    for (size_t r = 0; r < s->reps.size(); ++r) {
        const HostRep &R = s->reps[r];
        const size_t base = s->rep_pbase[r], n = R.type.size();
        std::memcpy(x3 + 3 * base, R.pos.data(), sizeof(float) * 3 * n);
        std::memcpy(v3 + 3 * base, R.vel.data(), sizeof(float) * 3 * n);
        std::memcpy(c + base * ns, R.conc.data(), sizeof(float) * n * ns);
    }
    return init_device(s, true);
}

// Pick the lanes per particle of the pair kernel by timing its forces-only
// mode (idempotent apart from the next binning's counters) for each choice,
// then rebuild the state with the winner.
// Size the neighbour lists of the current lane count from a counting pass
// over the sorted state in buffer 1 (capacity: 1.5 x the longest lane list,
// plus 16), allocate them and build them.
tdpd_status prepare_list(tdpd_sys *s)
{
    cudaStream_t st = exec_stream(s);
    const size_t lanes = (size_t)s->N * s->lpp;
    launch_list_build(list_args(s, s->buf[1], s->rb_all, 0), st);
    std::vector<int> cnt(lanes);
    CU(cudaMemcpyAsync(cnt.data(), s->nlc, sizeof(int) * lanes, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    int mx = 0;
    for (int c : cnt) mx = std::max(mx, c);
    const int cap = (mx * 3 / 2 + 16 + 7) / 8 * 8;
    const size_t need = (lanes + 31) / 32 * 32 * (size_t)cap;
    if (need > s->nl_ints) {
        if (s->nl) CU(cudaFree(s->nl));
        s->nl = nullptr;
        s->nl_ints = 0;
        cudaError_t e = cudaMalloc(&s->nl, need * sizeof(int));
        if (e != cudaSuccess) return fail(s, TDPD_ENOMEM, "neighbour lists (%zu bytes): %s", need * sizeof(int), cudaGetErrorString(e));
        s->nl_ints = need;
    }
    s->nl_cap = cap;
    launch_list_build(list_args(s, s->buf[1], s->rb_all, cap), st);
    CU(cudaGetLastError());
    return TDPD_OK;
}

// len steps from buffer p captured as one graph (with ev, event nodes around
// each kernel, all on one stream)
tdpd_status capture(tdpd_sys *s, int p, int len, cudaGraphExec_t *out, cudaEvent_t *ev = nullptr);

// Pick the pair kernel's shape at commit by timing its forces-only mode
// (idempotent apart from the next binning's counters) for each candidate:
// the lanes per particle (1..32, or the pinned count) and, with neighbour
// lists, the full shell (every pair from both sides) against the half shell
// (each pair once, partner shares by fixed-point atomics), unless the mode is
// pinned. The fastest of five timed launches per candidate; the candidates
// within 10 % of the best are then timed as 16-step graph replays; the first
// within 3 % of the best of those, half shell before full and fewer lanes
// before more (they are no slower once the caches are cold, and near-equal
// times would otherwise flip between runs). The state is then rebuilt with
// the winner.
// The host's state loaded again with lists sized for it and the current lane
// count: first sorted without lists (cell mode), so that the counting pass
// of prepare_list sees the state that is then loaded (a state stepped
// meanwhile may need shorter lists than the host's).
tdpd_status reload_state(tdpd_sys *s)
{
    tdpd_status rc;
    if (s->use_list) {
        s->use_list = false;
        rc = init_state(s);
        s->use_list = true;
        if (rc || (rc = prepare_list(s))) return rc;
    }
    return init_state(s);
}

tdpd_status autotune(tdpd_sys *s)
{
    cudaStream_t st = exec_stream(s);
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    std::vector<int> modes;
    if (!s->use_list) modes = {1};
    else if (s->mode_fixed) modes = {s->mode_fixed};
    else modes = {2, 1};
    struct Cand { int mode, lpp; float ms; };
    std::vector<Cand> t;
    for (int mode : modes) {
        for (int lpp = 1; lpp <= 32; lpp *= 2) {
            if (s->lanes_fixed > 0 && lpp != s->lanes_fixed) continue;
            if (s->lanes_fixed == 0 && lpp > 1 && (long)s->N * lpp > 4000000L) break;
            s->lpp = lpp;
            s->half = mode == 2;
            tdpd_status rc;
            if (s->use_list && (rc = prepare_list(s))) return rc;
            const PairArgs a = pair_args(s, s->buf[1], 0, s->tile_sum[1], s->disp[1]);
            launch_pair(a, st);                       // warm-up
            float fastest = 1e30f;
            for (int k = 0; k < 5; ++k) {
                cudaEventRecord(e0, st);
                launch_pair(a, st);
                cudaEventRecord(e1, st);
                cudaError_t e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return fail(s, TDPD_ECUDA, "autotune: %s", cudaGetErrorString(e));
                }
                fastest = std::min(fastest, ms);
            }
            t.push_back({mode, lpp, fastest});
        }
    }
    float best = 1e30f;
    for (const auto &x : t) best = std::min(best, x.ms);
    // the candidates within 10 % of the fastest launch are timed again as
    // whole steps (16 of them as one graph replay, after one warm-up replay),
    // which is what they will run as: in a short step the launch alone
    // misjudges the half shell's finishing pass and the membrane join
    std::vector<Cand> fin;
    for (const auto &x : t)
        if (x.ms <= 1.10f * best) fin.push_back(x);
    if (fin.size() > 1) {
        constexpr int STEPS = 16;
        float bstep = 1e30f;
        for (Cand &x : fin) {
            s->lpp = x.lpp;
            s->half = x.mode == 2;
            tdpd_status rc;
            if ((rc = reload_state(s))) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return rc;
            }
            cudaGraphExec_t g = nullptr;
            if ((rc = capture(s, s->parity, STEPS, &g))) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return rc;
            }
            cudaError_t e = cudaGraphLaunch(g, st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = cudaGraphLaunch(g, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&x.ms, e0, e1);
            cudaGraphExecDestroy(g);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return fail(s, TDPD_ECUDA, "autotune: %s", cudaGetErrorString(e));
            }
            bstep = std::min(bstep, x.ms);
        }
        t = fin;
        best = bstep;
        s->step = 0;
        if (s->builds) CU(cudaMemsetAsync(s->builds, 0, sizeof(uint32_t) * s->reps.size(), st));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    Cand win = t.empty() ? Cand{s->half ? 2 : 1, s->lpp, 0.f} : t.back();
    for (const auto &x : t)
        if (x.ms <= 1.03f * best) { win = x; break; }
    s->lpp = win.lpp;
    s->half = s->use_list && win.mode == 2;
    if (fin.size() > 1) return reload_state(s);      // buffer 1 holds a later state
    tdpd_status rc;
    if (s->use_list && (rc = prepare_list(s))) return rc;
    return init_state(s);
}

tdpd_status capture(tdpd_sys *s, int p, int len, cudaGraphExec_t *out, cudaEvent_t *ev)
{
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < len; ++k) enqueue_step(s, (p + k) & 1, s->cap, ev);
    cudaError_t e = cudaStreamEndCapture(s->cap, &g);
    if (e == cudaSuccess) e = cudaGetLastError();   // a launch or event record refused during capture
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(s, TDPD_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(s, TDPD_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return TDPD_OK;
}

// The loaded-state graph and the step graphs (both parities); graphs of an
// earlier capture (a changed list capacity) are replaced.
tdpd_status capture_graphs(tdpd_sys *s)
{
    tdpd_status rc;
    for (int p = 0; p < 2; ++p) {
        if (s->g1[p]) cudaGraphExecDestroy(s->g1[p]);
        if (s->glong[p]) cudaGraphExecDestroy(s->glong[p]);
        if (s->gtimed[p]) cudaGraphExecDestroy(s->gtimed[p]);
        s->g1[p] = s->glong[p] = s->gtimed[p] = nullptr;
    }
    if (s->ginit) cudaGraphExecDestroy(s->ginit);
    s->ginit = nullptr;
    {
        cudaGraph_t g;
        CU(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
        enqueue_init(s, s->cap, true);
        cudaError_t e = cudaStreamEndCapture(s->cap, &g);
        if (e != cudaSuccess) return fail(s, TDPD_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&s->ginit, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(s, TDPD_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    for (int p = 0; p < 2; ++p) {
        if ((rc = capture(s, p, 1, &s->g1[p]))) return rc;
        if ((rc = capture(s, p, GRAPH_LONG, &s->glong[p]))) return rc;
        if ((rc = capture(s, p, 1, &s->gtimed[p], s->ev))) return rc;
    }
    return TDPD_OK;
}

// Cell grids of every replica for a neighbour-list skin and a stencil width
// m_force (0: each replica's configured cells_per_cutoff, 2 by default):
// cells of edge >= (rcut + skin)/m; a periodic axis needs 2m+1 distinct
// cells, and a list partner must stay the nearest image (rcut + 2 skin <=
// L/2), so small boxes get a smaller skin. Sets each replica's m, skin and
// nc and returns the replica tables and the total cell count.
tdpd_status layout(tdpd_sys *s, float skin, int m_force, std::vector<RepParams> &P, int &NC)
{
    P.clear();
    long total = 0;
    for (size_t r = 0; r < s->reps.size(); ++r) {
        HostRep &R = s->reps[r];
        const float rcut = std::max(R.cfg.rc, R.cfg.rcc);
        R.m = m_force > 0 ? m_force : (R.cfg.cells_per_cutoff > 0 ? R.cfg.cells_per_cutoff : 2);
        float sk = s->use_list ? skin : 0.0f;
        for (int c = 0; c < 3; ++c) {
            const double L = R.cfg.L[c];
            if (R.cfg.periodic[c]) sk = std::min(sk, (float)(0.999 * (0.5 * L - rcut) / 2));
            sk = std::min(sk, (float)(0.999 * (L * R.m / ((2 * R.m + 1) * 1.0001) - rcut)));
        }
        R.skin = std::max(sk, 0.0f);
        for (int c = 0; c < 3; ++c) {
            R.nc[c] = (int)std::floor((double)R.cfg.L[c] * R.m / ((double)(rcut + R.skin) * 1.0001));
            if (R.nc[c] < 2 * R.m + 1) return fail(s, TDPD_EINVAL, "replica %zu: too few cells", r);
        }
        const long ncells = (long)R.nc[0] * R.nc[1] * R.nc[2];
        if (total + ncells > (1L << 30)) return fail(s, TDPD_EOVERFLOW, "too many cells");
        P.push_back(make_params(R, (int)total, s->rep_pbase[r], (int)R.type.size()));
        total += ncells;
    }
    NC = (int)total;
    return TDPD_OK;
}

// A list shape the commit may time: neighbour-list skin and stencil width.
struct Shape {
    float skin;
    int m;
};

// The shapes timed at commit, the default first: with neighbour lists, lanes
// that are not pinned and no skin set, the skins 0.15-0.4; with no replica
// pinning its cells_per_cutoff, the widths 2 and 3. Empty: nothing to time.
std::vector<Shape> shape_candidates(const tdpd_sys *s)
{
    std::vector<Shape> v;
    if (!s->use_list || s->lanes_fixed > 0) return v;
    bool tune_m = true;
    for (const HostRep &R : s->reps)
        if (R.cfg.cells_per_cutoff > 0) tune_m = false;
    const bool tune_skin = s->skin < 0.0f;
    if (!tune_m && !tune_skin) return v;
    const float skins_all[] = {DEFAULT_SKIN, 0.15f, 0.25f, 0.3f, 0.4f};
    std::vector<float> skins = tune_skin ? std::vector<float>(std::begin(skins_all), std::end(skins_all))
                                         : std::vector<float>{s->skin};
    std::vector<int> ms = tune_m ? std::vector<int>{2, 3} : std::vector<int>{0};
    for (int m : ms)
        for (float sk : skins) v.push_back({sk, m});
    return v;
}

// Make shape (skin, m) current: replica tables, cell count, lists sized and
// built for the state the host holds, forces evaluated.
tdpd_status apply_shape(tdpd_sys *s, const Shape &sh)
{
    std::vector<RepParams> P;
    int NC = 0;
    tdpd_status rc = layout(s, sh.skin, sh.m, P, NC);
    if (rc) return rc;
    if (NC > s->n_tiles * SCAN_TILE) return fail(s, TDPD_ESTATE, "cell arrays too small for a tuned shape");
    s->NC = NC;
    if ((rc = upload(s, s->d_reps, P.data(), P.size()))) return rc;
    return reload_state(s);
}

// Time the candidate shapes over a few whole steps each (the list rebuilds
// they cause included) with the default lanes and pair mode, keep the first
// within 3 % of the fastest (the default first), and leave it applied at
// step 0 with the host's state loaded.
tdpd_status tune_shape(tdpd_sys *s, const std::vector<Shape> &shapes)
{
    constexpr int STEPS = 16;
    cudaStream_t st = exec_stream(s);
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    std::vector<float> t(shapes.size(), 1e30f);
    tdpd_status rc = TDPD_OK;
    for (size_t k = 0; k < shapes.size() && !rc; ++k) {
        if ((rc = apply_shape(s, shapes[k]))) break;
        int p = s->parity;
        enqueue_step(s, p, st);                   // warm-up
        p ^= 1;
        cudaEventRecord(e0, st);
        for (int it = 0; it < STEPS; ++it, p ^= 1) enqueue_step(s, p, st);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t[k], e0, e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) rc = fail(s, TDPD_ECUDA, "shape tuning: %s", cudaGetErrorString(e));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const float best = *std::min_element(t.begin(), t.end());
    size_t win = 0;
    while (t[win] > 1.03f * best) ++win;
    s->shape_ms.assign(t.begin(), t.end());
    s->shape_win = (int)win;
    s->shape.skin = shapes[win].skin;
    s->shape.m = shapes[win].m;
    s->step = 0;
    if ((rc = apply_shape(s, shapes[win]))) return rc;
    if (s->builds) CU(cudaMemsetAsync(s->builds, 0, sizeof(uint32_t) * s->reps.size(), st));
    return TDPD_OK;
}

// List mode: the sort of a step as one cluster launch or as the kernel chain.
// Both give the same bits; unless the caller pinned one, time 16 steps of
// each as one graph replay (after one warm-up replay) and keep the cluster
// unless the chain is more than 3 % faster; then reload the host's state.
tdpd_status tune_sort(tdpd_sys *s)
{
    s->sort_ctas = 0;
    s->sort_ms.clear();
    if (!s->use_list || s->sort_fixed == 1) return TDPD_OK;
    int ctas = s->NC <= SORT_SMALL_MAX_NC ? sort_small_ctas(s->ns) : 0;
    const int max_n = ctas * SORT_SMALL_THREADS * SORT_SMALL_ITEMS;
    if (s->N > max_n) ctas = 0;
    if (s->sort_fixed == 2) {
        if (!ctas)
            return fail(s, TDPD_EINVAL, "the one-cluster sort needs at most %d particles and %d cells (here %d, %d) "
                        "and a resident cluster of 8 or 16 CTAs", 16 * SORT_SMALL_THREADS * SORT_SMALL_ITEMS,
                        SORT_SMALL_MAX_NC, s->N, s->NC);
        s->sort_ctas = ctas;
        return TDPD_OK;
    }
    if (!ctas) return TDPD_OK;
    constexpr int STEPS = 16;
    cudaStream_t st = exec_stream(s);
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float t[2] = {1e30f, 1e30f};
    tdpd_status rc = TDPD_OK;
    for (int k = 0; k < 2 && !rc; ++k) {
        s->sort_ctas = k == 0 ? ctas : 0;
        cudaGraphExec_t g = nullptr;
        if ((rc = capture(s, s->parity, STEPS, &g))) break;
        cudaError_t e = cudaGraphLaunch(g, st);            // warm-up (an even count: same parity after)
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = cudaGraphLaunch(g, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t[k], e0, e1);
        cudaGraphExecDestroy(g);
        if (e != cudaSuccess) rc = fail(s, TDPD_ECUDA, "sort tuning: %s", cudaGetErrorString(e));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    s->sort_ms.assign(t, t + 2);
    s->sort_ctas = t[0] <= 1.03f * t[1] ? ctas : 0;
    s->step = 0;
    if ((rc = init_state(s))) return rc;
    if (s->builds) CU(cudaMemsetAsync(s->builds, 0, sizeof(uint32_t) * s->reps.size(), st));
    return TDPD_OK;
}

tdpd_status commit(tdpd_sys *s)
{
    if (s->committed) return TDPD_OK;
    if (s->reps.empty()) return fail(s, TDPD_ESTATE, "no replicas");
    s->ns = s->reps[0].cfg.n_species;
    int N = 0, NC = 0;
    const float skin = s->skin < 0.0f ? DEFAULT_SKIN : s->skin;
    s->use_list = skin > 0.0f;
    s->rep_pbase.clear();
    s->rep_rbc0.clear();
    s->h_rbcs.clear();
    s->topos.clear();
    std::vector<RepParams> P;
    std::vector<float> a0j;
    std::vector<float2> bond;
    int max_nv = 0;
    for (size_t r = 0; r < s->reps.size(); ++r) {
        HostRep &R = s->reps[r];
        if (R.cfg.n_species != s->ns) return fail(s, TDPD_EINVAL, "replica %zu: all replicas need the same number of species", r);
        const int n = (int)R.type.size();
        if (n > TDPD_MAX_IDS) return fail(s, TDPD_EOVERFLOW, "replica %zu: %d particles exceed %d", r, n, TDPD_MAX_IDS);
        const float rcut = std::max(R.cfg.rc, R.cfg.rcc);
        for (int c = 0; c < 3; ++c)
            if ((double)R.cfg.L[c] < 3.0 * rcut * 1.0001)
                return fail(s, TDPD_EINVAL, "replica %zu: box edge %g is shorter than 3 cut-offs (%g)", r, R.cfg.L[c], rcut);
        if (!R.rbcs.empty() && !R.has_mem) return fail(s, TDPD_ESTATE, "replica %zu has membranes but no tdpd_set_membrane", r);
        {
            // Eq. 4: sigma^2 = 2 kT gamma with one temperature for every type
            // pair that has a dissipative or random force
            double kT = -1.0;
            for (int i = 0; i < R.cfg.n_types; ++i)
                for (int j = i; j < R.cfg.n_types; ++j) {
                    const double g = R.gamma[i * MAXT + j], sg = R.sigma[i * MAXT + j];
                    if (g == 0.0 && sg == 0.0) continue;
                    if (g == 0.0 || sg == 0.0)
                        return fail(s, TDPD_EINVAL, "replica %zu, types %d-%d: Eq. 4 needs gamma and sigma both zero or both positive", r, i, j);
                    const double t = sg * sg / (2.0 * g);
                    if (kT < 0.0) kT = t;
                    else if (std::fabs(t - kT) > 1e-5 * kT)
                        return fail(s, TDPD_EINVAL, "replica %zu, types %d-%d: sigma^2 / (2 gamma) = %g differs from %g (Eq. 4 fixes one kT)", r, i, j, t, kT);
                }
        }
        s->rep_pbase.push_back(N);
        s->rep_rbc0.push_back((int)s->h_rbcs.size());
        // membranes
        int first = R.n_free;
        for (size_t b = 0; b < R.rbcs.size(); ++b) {
            const HostRbc &H = R.rbcs[b];
            int ti = -1;
            for (size_t t = 0; t < s->topos.size(); ++t)
                if (s->topos[t].nv == H.nv && s->topos[t].tri == H.tri) { ti = (int)t; break; }
            if (ti < 0) {
                Topo T;
                tdpd_status rc = build_topo(s, H.nv, H.ntri, H.tri.data(), T);
                if (rc) return rc;
                s->topos.push_back(std::move(T));
                ti = (int)s->topos.size() - 1;
            }
            const Topo &T = s->topos[ti];
            RbcDev D{};
            D.gbase = N + first;
            D.rep = (int)r;
            D.topo = ti;
            D.nv = H.nv;
            D.ntri = H.ntri;
            D.ne = T.ne;
            D.a0j_off = (int)a0j.size();
            D.bond_off = (int)bond.size();
            std::vector<double> x;
            unwrap(R, T, H.rest.data(), x);
            double A = 0, V = 0;
            for (int t = 0; t < H.ntri; ++t) {
                const double *p0 = &x[3 * H.tri[3 * t]], *p1 = &x[3 * H.tri[3 * t + 1]], *p2 = &x[3 * H.tri[3 * t + 2]];
                double u[3], w[3], n3[3], c12[3];
                for (int k = 0; k < 3; ++k) { u[k] = p1[k] - p0[k]; w[k] = p2[k] - p0[k]; }
                n3[0] = u[1] * w[2] - u[2] * w[1];
                n3[1] = u[2] * w[0] - u[0] * w[2];
                n3[2] = u[0] * w[1] - u[1] * w[0];
                c12[0] = p1[1] * p2[2] - p1[2] * p2[1];
                c12[1] = p1[2] * p2[0] - p1[0] * p2[2];
                c12[2] = p1[0] * p2[1] - p1[1] * p2[0];
                const double At = 0.5 * std::sqrt(n3[0] * n3[0] + n3[1] * n3[1] + n3[2] * n3[2]);
                a0j.push_back((float)At);
                A += At;
                V += (p0[0] * c12[0] + p0[1] * c12[1] + p0[2] * c12[2]) / 6.0;
            }
            const tdpd_membrane &m = R.mem;
            const double x0 = m.x0;
            const double fw = (double)m.kT / m.p * (0.25 / ((1 - x0) * (1 - x0)) - 0.25 + x0);
            for (int e = 0; e < T.ne; ++e) {
                const int i = T.edges[e].first, j = T.edges[e].second;
                double d2 = 0;
                for (int k = 0; k < 3; ++k) d2 += (x[3 * i + k] - x[3 * j + k]) * (x[3 * i + k] - x[3 * j + k]);
                const double l0 = std::sqrt(d2);
                bond.push_back(make_float2((float)(l0 / x0), (float)(fw * std::pow(l0, (double)m.m))));
            }
            D.A0 = A;
            D.V0 = m.v_ratio > 0 ? (double)m.v_ratio * std::pow(A, 1.5) : V;
            D.kgA0 = (double)m.kg / D.A0;
            D.kvV0 = (double)m.kv / D.V0;
            D.inv_nv = 1.0 / H.nv;
            s->h_rbcs.push_back(D);
            max_nv = std::max(max_nv, H.nv);
            first += H.nv;
        }
        N += n;
    }
    s->N = N;
    // the cell grids of the default shape; with the shape tuned at commit the
    // cell arrays are sized for the candidate with the most cells
    tdpd_status lrc = layout(s, skin, 0, P, NC);
    if (lrc) return lrc;
    s->NC = NC;
    s->shape.skin = s->use_list ? skin : 0.0f;
    s->shape.m = 0;
    const std::vector<Shape> shapes = shape_candidates(s);
    int NC_alloc = NC;
    for (const Shape &sh : shapes) {
        std::vector<RepParams> Q;
        int nc2 = 0;
        if ((lrc = layout(s, sh.skin, sh.m, Q, nc2))) return lrc;
        NC_alloc = std::max(NC_alloc, nc2);
    }
    if (!shapes.empty() && (lrc = layout(s, skin, 0, P, NC))) return lrc;
    s->n_tiles = (NC_alloc + SCAN_TILE - 1) / SCAN_TILE;
    s->h_chunks.clear();
    for (size_t r = 0; r < s->reps.size(); ++r) {
        const int b0 = s->rep_pbase[r], n = (int)s->reps[r].type.size();
        for (int k = 0; k < n || k == 0; k += OBS_CHUNK)
            s->h_chunks.push_back(make_int4((int)r, b0 + k, b0 + std::min(n, k + OBS_CHUNK), 0));
    }
    // lanes per particle: enough threads to fill the GPU (~300k resident)
    s->lpp = 1;
    while (s->lpp < 8 && (long)N * s->lpp < 300000) s->lpp *= 2;
    s->n_rbc = (int)s->h_rbcs.size();
    s->all_lagged = s->n_rbc > 0;
    for (const HostRep &R : s->reps)
        if (!R.rbcs.empty() && !R.mem.lagged_av) s->all_lagged = false;
    s->max_nv = max_nv;
    if (N == 0) return fail(s, TDPD_ESTATE, "no particles loaded");

    // device allocations
    tdpd_status rc;
    const int ns = s->ns;
    for (int p = 0; p < 2; ++p) {
        Buffers &B = s->buf[p];
        if ((rc = dalloc(s, &B.pos, N)) || (rc = dalloc(s, &B.vt, N)) || (rc = dalloc(s, &B.vel, N)) ||
            (rc = dalloc(s, &B.frc, N)) || (rc = dalloc(s, &B.C, (size_t)N * ns)) ||
            (rc = dalloc(s, &B.Ct, (size_t)N * ns)) || (rc = dalloc(s, &B.Q, (size_t)N * ns)))
            return rc;
    }
    if ((rc = dalloc(s, &s->fext, N)) || (rc = dalloc(s, &s->mx, N)) || (rc = dalloc(s, &s->mv, N)) ||
        (rc = dalloc(s, &s->inv, N)) || (rc = dalloc(s, &s->cellrank, N)) ||
        (rc = dalloc(s, &s->keys, N)) || (rc = dalloc(s, &s->count, (size_t)s->n_tiles * SCAN_TILE)) ||
        (rc = dalloc(s, &s->cell_start, (size_t)s->n_tiles * SCAN_TILE + 1)) ||
        (rc = dalloc(s, &s->tile_sum[0], s->n_tiles)) || (rc = dalloc(s, &s->tile_sum[1], s->n_tiles)) ||
        (rc = dalloc(s, &s->d_chunks, s->h_chunks.size())) ||
        (rc = dalloc(s, &s->errw, s->reps.size())) || (rc = dalloc(s, &s->quar, s->reps.size())) ||
        (rc = dalloc(s, &s->step_ctr, 3)) ||
        (rc = dalloc(s, &s->d_reps, P.size())) || (rc = dalloc(s, &s->d_obs, OBS_K * s->h_chunks.size())))
        return rc;
    if ((rc = upload(s, s->d_reps, P.data(), P.size()))) return rc;
    if ((rc = upload(s, s->d_chunks, s->h_chunks.data(), s->h_chunks.size()))) return rc;
    {
        // the end of the last cell (and of the padding) is the particle count
        std::vector<int> tail((size_t)s->n_tiles * SCAN_TILE + 1 - NC, N);
        if ((rc = upload(s, s->cell_start + NC, tail.data(), tail.size()))) return rc;
    }
    if (s->n_rbc) {
        // per mesh: its triangles, and its fans at a fixed stride (the
        // largest degree) with each entry's cyclic neighbours
        std::vector<int> tri, t_tri(s->topos.size()), t_fan(s->topos.size()), t_stride(s->topos.size());
        std::vector<FanEntry> fan;
        for (size_t t = 0; t < s->topos.size(); ++t) {
            const Topo &T = s->topos[t];
            int mx = 0;
            for (int v = 0; v < T.nv; ++v) mx = std::max(mx, T.ring_off[v + 1] - T.ring_off[v]);
            t_tri[t] = (int)tri.size();
            t_fan[t] = (int)fan.size();
            t_stride[t] = mx;
            tri.insert(tri.end(), T.tri.begin(), T.tri.end());
            for (int v = 0; v < T.nv; ++v) {
                const int o = T.ring_off[v], deg = T.ring_off[v + 1] - o;
                for (int l = 0; l < mx; ++l) {
                    FanEntry F{-1, -1, -1, -1, -1, -1, 0, 0};
                    if (l < deg) {
                        const RingEntry &E = T.ring[o + l];
                        F = FanEntry{E.nb, E.edge, E.tri, E.across, T.ring[o + (l + 1) % deg].nb,
                                     T.ring[o + (l + deg - 1) % deg].nb, 0, 0};
                    }
                    fan.push_back(F);
                }
            }
        }
        for (RbcDev &D : s->h_rbcs) {
            D.tri_off = t_tri[D.topo];
            D.fan_off = t_fan[D.topo];
            D.fan_stride = t_stride[D.topo];
        }
        if ((rc = dalloc(s, &s->d_rbcs, s->n_rbc)) || (rc = dalloc(s, &s->d_tri, tri.size())) ||
            (rc = dalloc(s, &s->d_fan, fan.size())) || (rc = dalloc(s, &s->d_a0j, a0j.size())) ||
            (rc = dalloc(s, &s->d_bond, bond.size())) || (rc = dalloc(s, &s->d_ref[0], s->n_rbc)) ||
            (rc = dalloc(s, &s->d_ref[1], s->n_rbc)) || (rc = dalloc(s, &s->d_av[0], s->n_rbc)) ||
            (rc = dalloc(s, &s->d_av[1], s->n_rbc)) || (rc = dalloc(s, &s->d_cgv[0], s->n_rbc)) ||
            (rc = dalloc(s, &s->d_cgv[1], s->n_rbc)))
            return rc;
        if ((rc = upload(s, s->d_rbcs, s->h_rbcs.data(), s->n_rbc)) || (rc = upload(s, s->d_tri, tri.data(), tri.size())) ||
            (rc = upload(s, s->d_fan, fan.data(), fan.size())) || (rc = upload(s, s->d_a0j, a0j.data(), a0j.size())) ||
            (rc = upload(s, s->d_bond, bond.data(), bond.size())))
            return rc;
    }
    {
        s->h_stage_bytes = stage_bytes(N, ns);
        void *hp = nullptr;
        CU(cudaMallocHost(&hp, s->h_stage_bytes));
        s->h_stage = static_cast<unsigned char *>(hp);
        s->h_obs = reinterpret_cast<double *>(s->h_stage);
        CU(cudaEventCreateWithFlags(&s->stage_done, cudaEventDisableTiming));
        if ((rc = dalloc(s, &s->d_obs_tot, OBS_K)) || (rc = dalloc(s, &s->d_obs_done, 1)) || (rc = dalloc(s, &s->d_in, (size_t)N * (6 + ns))) ||
            (rc = dalloc(s, &s->d_wstat, N)) || (rc = dalloc(s, &s->d_flag, 1)))
            return rc;
        std::vector<int4> ws(N);
        int rb0 = 0;
        for (size_t r = 0; r < s->reps.size(); ++r) {
            const HostRep &R = s->reps[r];
            for (size_t i = 0; i < R.type.size(); ++i)
                ws[s->rep_pbase[r] + i] = make_int4((int)((uint32_t)i | ((uint32_t)R.type[i] << 24)), (int)r,
                                                    R.body[i] >= 0 ? rb0 + R.body[i] : -1, 0);
            rb0 += (int)R.rbcs.size();
        }
        if ((rc = upload(s, s->d_wstat, ws.data(), N))) return rc;
        CU(cudaMemsetAsync(s->d_obs_done, 0, sizeof(unsigned), exec_stream(s)));
    }
    if (s->use_list) {
        const int nrep = (int)s->reps.size();
        if ((rc = dalloc(s, &s->xb, N)) || (rc = dalloc(s, &s->disp[0], nrep)) || (rc = dalloc(s, &s->disp[1], nrep)) ||
            (rc = dalloc(s, &s->rb, nrep + 1)) || (rc = dalloc(s, &s->rb_all, nrep + 1)) ||
            (rc = dalloc(s, &s->nlc, (size_t)N * 32)) || (rc = dalloc(s, &s->builds, nrep)))
            return rc;
        CU(cudaMemsetAsync(s->builds, 0, sizeof(uint32_t) * nrep, exec_stream(s)));
        // half-shell accumulators (zero between steps) and own sums
        if ((rc = dalloc(s, &s->accF, (size_t)N * 4)) || (rc = dalloc(s, &s->accQ, (size_t)N * ns)) ||
            (rc = dalloc(s, &s->fown, N)) || (rc = dalloc(s, &s->qown, (size_t)N * ns)))
            return rc;
        CU(cudaMemsetAsync(s->accF, 0, sizeof(long long) * 4 * (size_t)N, exec_stream(s)));
        CU(cudaMemsetAsync(s->accQ, 0, sizeof(long long) * (size_t)N * ns, exec_stream(s)));
        std::vector<uint32_t> ones(nrep + 1, 1u);
        if ((rc = upload(s, s->rb_all, ones.data(), ones.size()))) return rc;
        CU(cudaMemsetAsync(s->disp[0], 0, sizeof(uint32_t) * nrep, exec_stream(s)));
        CU(cudaMemsetAsync(s->disp[1], 0, sizeof(uint32_t) * nrep, exec_stream(s)));
    }
    s->step = 0;
    if (s->lanes_fixed > 0) s->lpp = s->lanes_fixed;
    // pinned lanes and no pinned mode: the half shell, without timing
    s->half = s->use_list && s->mode_fixed != 1;
    if (s->use_list) {
        // a sorted state for the counting pass that sizes the lists
        s->use_list = false;
        rc = init_state(s);
        s->use_list = true;
        if (rc || (rc = prepare_list(s))) return rc;
    }
    if ((rc = init_state(s))) return rc;
    CU(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&s->join, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&s->gathered, cudaEventDisableTiming));
    if (!shapes.empty() && (rc = tune_shape(s, shapes))) return rc;
    if (s->lanes_fixed == 0 && (rc = autotune(s))) return rc;
    if ((rc = tune_sort(s))) return rc;
    const int nk = (int)step_kernels(s).size();
    for (int k = 0; k <= nk; ++k) CU(cudaEventCreate(&s->ev[k]));
    s->n_ev = nk + 1;
    if ((rc = capture_graphs(s))) return rc;
    CU(cudaStreamSynchronize(exec_stream(s)));
    s->committed = true;
    return TDPD_OK;
}

tdpd_status ensure(tdpd_sys *s)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    return s->committed ? TDPD_OK : commit(s);
}

HostRep *rep_of(tdpd_sys *s, int r)
{
    if (r < 0 || r >= (int)s->reps.size()) return nullptr;
    return &s->reps[r];
}

// Download the current sorted state of replica r into load order.
tdpd_status download(tdpd_sys *s, int r, float *pos, float *vel, float *conc, float *frc, float *flux)
{
    cudaStream_t st = exec_stream(s);
    const HostRep &R = s->reps[r];
    const int n = (int)R.type.size(), base = s->rep_pbase[r], ns = s->ns;
    std::vector<int> inv(n);
    std::vector<float4> a(n), b(n);
    std::vector<float> c((size_t)n * ns), q((size_t)n * ns);
    const Buffers &B = s->buf[s->parity];
    CU(cudaMemcpyAsync(inv.data(), s->inv + base, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    // the replica's slots are the contiguous range [base, base+n)
    if (pos) CU(cudaMemcpyAsync(a.data(), B.pos + base, sizeof(float4) * n, cudaMemcpyDeviceToHost, st));
    if (vel) CU(cudaMemcpyAsync(b.data(), B.vel + base, sizeof(float4) * n, cudaMemcpyDeviceToHost, st));
    if (conc) CU(cudaMemcpyAsync(c.data(), B.C + (size_t)base * ns, sizeof(float) * n * ns, cudaMemcpyDeviceToHost, st));
    std::vector<float4> f(frc ? n : 0);
    if (frc) CU(cudaMemcpyAsync(f.data(), B.frc + base, sizeof(float4) * n, cudaMemcpyDeviceToHost, st));
    if (flux) CU(cudaMemcpyAsync(q.data(), B.Q + (size_t)base * ns, sizeof(float) * n * ns, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) {
        const int k = inv[i] - base;
        if (k < 0 || k >= n) return fail(s, TDPD_ESTATE, "corrupt slot map");
        if (pos) { pos[3 * i] = a[k].x; pos[3 * i + 1] = a[k].y; pos[3 * i + 2] = a[k].z; }
        if (vel) { vel[3 * i] = b[k].x; vel[3 * i + 1] = b[k].y; vel[3 * i + 2] = b[k].z; }
        if (frc) { frc[3 * i] = f[k].x; frc[3 * i + 1] = f[k].y; frc[3 * i + 2] = f[k].z; }
        for (int sp = 0; sp < ns; ++sp) {
            if (conc) conc[(size_t)i * ns + sp] = c[(size_t)k * ns + sp];
            if (flux) flux[(size_t)i * ns + sp] = q[(size_t)k * ns + sp];
        }
    }
    return TDPD_OK;
}

tdpd_status check_config(tdpd_sys *s, const tdpd_config *c)
{
    if (!c) return fail(s, TDPD_EINVAL, "null config");
    char msg[160];
    if (config_error(*c, msg, sizeof msg)) return fail(s, TDPD_EINVAL, "%s", msg);
    return TDPD_OK;
}

}  // namespace

extern "C" {

tdpd_status tdpd_create(tdpd_sys **out, const tdpd_config *cfg)
{
    if (!out) return fail(nullptr, TDPD_EINVAL, "null output handle");
    *out = nullptr;
    tdpd_status rc = check_config(nullptr, cfg);
    if (rc) return rc;
    tdpd_sys *s = new (std::nothrow) tdpd_sys;
    if (!s) return fail(nullptr, TDPD_ENOMEM, "host allocation failed");
    s->reps.emplace_back();
    s->reps[0].cfg = *cfg;
    cudaError_t e = cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        fail(nullptr, TDPD_ECUDA, "stream creation: %s", cudaGetErrorString(e));
        delete s;
        return TDPD_ECUDA;
    }
    *out = s;
    return TDPD_OK;
}

tdpd_status tdpd_set_pair(tdpd_sys *s, int ti, int tj, float a, float gamma, float sigma)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed) return fail(s, TDPD_ESTATE, "parameters are fixed after commit");
    HostRep &R = s->reps[0];
    if (s->reps.size() != 1) return fail(s, TDPD_ESTATE, "set parameters on the replicas before batching");
    if (ti < 0 || tj < 0 || ti >= R.cfg.n_types || tj >= R.cfg.n_types) return fail(s, TDPD_EINVAL, "type out of range");
    if (!std::isfinite(a) || !(gamma >= 0) || !(sigma >= 0) || !std::isfinite(gamma) || !std::isfinite(sigma))
        return fail(s, TDPD_EINVAL, "bad pair coefficients");
    for (int k = 0; k < 2; ++k) {
        const int i = k ? tj : ti, j = k ? ti : tj;
        R.a[i * MAXT + j] = a;
        R.gamma[i * MAXT + j] = gamma;
        R.sigma[i * MAXT + j] = sigma;
    }
    return TDPD_OK;
}

tdpd_status tdpd_set_kappa(tdpd_sys *s, int ti, int tj, int sp, float kappa)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed || s->reps.size() != 1) return fail(s, TDPD_ESTATE, "parameters are fixed after commit or batching");
    HostRep &R = s->reps[0];
    if (ti < 0 || tj < 0 || ti >= R.cfg.n_types || tj >= R.cfg.n_types || sp < 0 || sp >= R.cfg.n_species)
        return fail(s, TDPD_EINVAL, "type or species out of range");
    if (!(kappa >= 0) || !std::isfinite(kappa)) return fail(s, TDPD_EINVAL, "kappa must be finite and >= 0");
    R.kappa[(ti * MAXT + tj) * MAXS + sp] = kappa;
    R.kappa[(tj * MAXT + ti) * MAXS + sp] = kappa;
    return TDPD_OK;
}

tdpd_status tdpd_set_reaction(tdpd_sys *s, float k, int src, int dst, uint32_t types)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed || s->reps.size() != 1) return fail(s, TDPD_ESTATE, "parameters are fixed after commit or batching");
    HostRep &R = s->reps[0];
    if (src < 0 || dst < 0 || src >= R.cfg.n_species || dst >= R.cfg.n_species || src == dst)
        return fail(s, TDPD_EINVAL, "reaction species out of range");
    if (!std::isfinite(k)) return fail(s, TDPD_EINVAL, "reaction rate must be finite");
    R.k_react = k;
    R.r_src = src;
    R.r_dst = dst;
    R.r_types = types;
    return TDPD_OK;
}

tdpd_status tdpd_set_random_flux(tdpd_sys *s, float m_s, float rho)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed || s->reps.size() != 1) return fail(s, TDPD_ESTATE, "parameters are fixed after commit or batching");
    if (!(m_s >= 0.0f && rho >= 0.0f && std::isfinite(m_s) && std::isfinite(rho)))
        return fail(s, TDPD_EINVAL, "random flux: m_s and rho must be finite and >= 0");
    s->reps[0].qr_ms = m_s;
    s->reps[0].qr_rho = rho;
    return TDPD_OK;
}

tdpd_status tdpd_set_body_force_profile(tdpd_sys *s, int mode)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed || s->reps.size() != 1) return fail(s, TDPD_ESTATE, "parameters are fixed after commit or batching");
    if (mode != 0 && mode != 1) return fail(s, TDPD_EINVAL, "body force profile must be 0 or 1");
    s->reps[0].fbody_flip = mode;
    return TDPD_OK;
}

tdpd_status tdpd_set_cylinder_wall(tdpd_sys *s, float radius)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed || s->reps.size() != 1) return fail(s, TDPD_ESTATE, "parameters are fixed after commit or batching");
    const tdpd_config &c = s->reps[0].cfg;
    if (!(radius >= 0.0f) || !std::isfinite(radius)) return fail(s, TDPD_EINVAL, "cylinder radius must be finite and >= 0");
    if (radius > 0.0f && (!c.periodic[1] || !c.periodic[2] || !(2.0f * radius < std::min(c.L[1], c.L[2]))))
        return fail(s, TDPD_EINVAL, "cylinder wall needs periodic y and z and a diameter below min(L_y, L_z)");
    s->reps[0].cyl_R = radius;
    return TDPD_OK;
}

tdpd_status tdpd_set_membrane(tdpd_sys *s, const tdpd_membrane *m)
{
    if (!s || !m) return fail(s, TDPD_EINVAL, "null argument");
    if (s->committed || s->reps.size() != 1) return fail(s, TDPD_ESTATE, "parameters are fixed after commit or batching");
    if (!(m->p > 0) || !(m->x0 > 0 && m->x0 < 1) || !(m->m > 0) || !(m->kT >= 0))
        return fail(s, TDPD_EINVAL, "membrane: need p > 0, 0 < x0 < 1, m > 0, kT >= 0");
    if (!(m->gammaT >= 0) || !(3.0f * m->gammaC >= m->gammaT))
        return fail(s, TDPD_EINVAL, "membrane: need gammaT >= 0 and 3 gammaC >= gammaT");
    s->reps[0].mem = *m;
    s->reps[0].has_mem = true;
    return TDPD_OK;
}

tdpd_status tdpd_add_particles(tdpd_sys *s, int n, const float *pos, const float *vel,
                               const float *conc, const int32_t *type)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed || s->reps.size() != 1) return fail(s, TDPD_ESTATE, "particles are fixed after commit or batching");
    HostRep &R = s->reps[0];
    if (!R.rbcs.empty()) return fail(s, TDPD_ESTATE, "add free particles before membranes");
    if (n < 0 || (n > 0 && (!pos || !vel || !type))) return fail(s, TDPD_EINVAL, "bad particle arrays");
    const int ns = R.cfg.n_species;
    if ((long)R.type.size() + n > TDPD_MAX_IDS) return fail(s, TDPD_EOVERFLOW, "more than %d particles", TDPD_MAX_IDS);
    for (int i = 0; i < n; ++i) {
        if (type[i] < 0 || type[i] >= R.cfg.n_types) return fail(s, TDPD_EINVAL, "particle %d: type %d out of range", i, type[i]);
        for (int c = 0; c < 3; ++c) {
            const float x = pos[3 * i + c];
            if (!(x >= 0.0f && x < R.cfg.L[c])) return fail(s, TDPD_EINVAL, "particle %d: coordinate %d = %g outside [0, L)", i, c, x);
            if (!std::isfinite(vel[3 * i + c])) return fail(s, TDPD_EINVAL, "particle %d: non-finite velocity", i);
        }
    }
    R.pos.insert(R.pos.end(), pos, pos + 3 * (size_t)n);
    R.vel.insert(R.vel.end(), vel, vel + 3 * (size_t)n);
    if (conc) R.conc.insert(R.conc.end(), conc, conc + (size_t)n * ns);
    else R.conc.insert(R.conc.end(), (size_t)n * ns, 0.0f);
    R.type.insert(R.type.end(), type, type + n);
    R.body.insert(R.body.end(), (size_t)n, -1);
    R.n_free += n;
    return TDPD_OK;
}

tdpd_status tdpd_add_rbc(tdpd_sys *s, int nv, const float *pos, const float *vel, const float *conc,
                         int type, int ntri, const int32_t *tri, const float *rest, int *rbc_index)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed || s->reps.size() != 1) return fail(s, TDPD_ESTATE, "membranes are fixed after commit or batching");
    HostRep &R = s->reps[0];
    if (nv < 4 || nv > 1024 || !pos || !vel || !tri || ntri != 2 * nv - 4)
        return fail(s, TDPD_EINVAL, "membrane needs 4..1024 vertices and 2*nv-4 triangles");
    if (type < 0 || type >= R.cfg.n_types) return fail(s, TDPD_EINVAL, "membrane type out of range");
    if ((long)R.type.size() + nv > TDPD_MAX_IDS) return fail(s, TDPD_EOVERFLOW, "more than %d particles", TDPD_MAX_IDS);
    for (int i = 0; i < 3 * nv; ++i) {
        const int c = i % 3;
        if (!(pos[i] >= 0.0f && pos[i] < R.cfg.L[c])) return fail(s, TDPD_EINVAL, "vertex %d outside [0, L)", i / 3);
    }
    Topo T;
    tdpd_status rc = build_topo(s, nv, ntri, tri, T);   // validate now
    if (rc) return rc;
    HostRbc H;
    H.nv = nv;
    H.ntri = ntri;
    H.type = type;
    H.tri.assign(tri, tri + 3 * ntri);
    H.rest.assign(rest ? rest : pos, (rest ? rest : pos) + 3 * (size_t)nv);
    const int b = (int)R.rbcs.size();
    const int ns = R.cfg.n_species;
    R.rbcs.push_back(std::move(H));
    R.pos.insert(R.pos.end(), pos, pos + 3 * (size_t)nv);
    R.vel.insert(R.vel.end(), vel, vel + 3 * (size_t)nv);
    if (conc) R.conc.insert(R.conc.end(), conc, conc + (size_t)nv * ns);
    else R.conc.insert(R.conc.end(), (size_t)nv * ns, 0.0f);
    R.type.insert(R.type.end(), (size_t)nv, type);
    R.body.insert(R.body.end(), (size_t)nv, b);
    if (rbc_index) *rbc_index = b;
    return TDPD_OK;
}

tdpd_status tdpd_batch_create(tdpd_sys **out, tdpd_sys *const *replicas, int n)
{
    if (!out || !replicas || n <= 0) return fail(nullptr, TDPD_EINVAL, "bad batch arguments");
    *out = nullptr;
    tdpd_sys *s = new (std::nothrow) tdpd_sys;
    if (!s) return fail(nullptr, TDPD_ENOMEM, "host allocation failed");
    for (int k = 0; k < n; ++k) {
        tdpd_sys *r = replicas[k];
        if (!r || r->reps.size() != 1) {
            delete s;
            return fail(nullptr, TDPD_EINVAL, "replica %d is not a single-replica handle", k);
        }
        HostRep R = r->reps[0];
        if (r->committed) {
            const int m = (int)R.type.size();
            tdpd_status rc = download(r, 0, R.pos.data(), R.vel.data(), R.conc.data(), nullptr, nullptr);
            if (rc) {
                delete s;
                return fail(nullptr, rc, "replica %d: %s", k, r->err.c_str());
            }
            (void)m;
            R.step = r->step;
        }
        s->reps.push_back(std::move(R));
    }
    cudaError_t e = cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return fail(nullptr, TDPD_ECUDA, "stream creation: %s", cudaGetErrorString(e));
    }
    *out = s;
    return TDPD_OK;
}

tdpd_status tdpd_set_stream(tdpd_sys *s, void *stream)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    s->user = (cudaStream_t)stream;
    return TDPD_OK;
}

tdpd_status tdpd_set_lanes(tdpd_sys *s, int lanes)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed) return fail(s, TDPD_ESTATE, "lanes are fixed after commit");
    if (lanes < 0 || lanes > 32 || (lanes & (lanes - 1)))
        return fail(s, TDPD_EINVAL, "lanes must be 0 (timed) or 1, 2, 4, 8, 16, 32");
    s->lanes_fixed = lanes;
    return TDPD_OK;
}

tdpd_status tdpd_list_shape(tdpd_sys *s, float *skin, int *cells_per_cutoff, float *tuning_ms, int max_tuning,
                            int *n_tuning)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    if (skin) *skin = s->shape.skin;
    if (cells_per_cutoff) *cells_per_cutoff = s->reps[0].m;
    const int n = (int)s->shape_ms.size();
    for (int k = 0; k < n && k < max_tuning && tuning_ms; ++k) tuning_ms[k] = s->shape_ms[k];
    if (n_tuning) *n_tuning = n;
    return TDPD_OK;
}

tdpd_status tdpd_set_pair_mode(tdpd_sys *s, int mode)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed) return fail(s, TDPD_ESTATE, "the pair mode is fixed after commit");
    if (mode < 0 || mode > 2) return fail(s, TDPD_EINVAL, "pair mode must be 0 (chosen at commit), 1 (full shell) or 2 (half shell)");
    s->mode_fixed = mode;
    return TDPD_OK;
}

int tdpd_pair_mode(const tdpd_sys *s)
{
    if (!s) return 0;
    if (!s->committed) return s->mode_fixed;
    return s->half ? 2 : 1;
}

tdpd_status tdpd_set_sort_mode(tdpd_sys *s, int mode)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed) return fail(s, TDPD_ESTATE, "the sort is fixed after commit");
    if (mode < 0 || mode > 2)
        return fail(s, TDPD_EINVAL, "sort mode must be 0 (chosen at commit), 1 (kernel chain) or 2 (one cluster)");
    s->sort_fixed = mode;
    return TDPD_OK;
}

int tdpd_sort_mode(const tdpd_sys *s, float *tuning_ms)
{
    if (!s) return 0;
    if (!s->committed) return s->sort_fixed;
    if (tuning_ms) {
        tuning_ms[0] = s->sort_ms.size() == 2 ? s->sort_ms[0] : -1.0f;
        tuning_ms[1] = s->sort_ms.size() == 2 ? s->sort_ms[1] : -1.0f;
    }
    return s->sort_ctas ? 2 : 1;
}

tdpd_status tdpd_set_skin(tdpd_sys *s, float skin)
{
    if (!s) return fail(nullptr, TDPD_EINVAL, "null handle");
    if (s->committed) return fail(s, TDPD_ESTATE, "the skin is fixed after commit");
    if (!(skin >= 0.0f && skin < 1e3f)) return fail(s, TDPD_EINVAL, "skin must be finite and >= 0");
    s->skin = skin;
    return TDPD_OK;
}

tdpd_status tdpd_commit(tdpd_sys *s) { return ensure(s); }

int tdpd_lanes(const tdpd_sys *s)
{
    if (!s) return 0;
    return s->committed ? s->lpp : s->lanes_fixed;
}

tdpd_status tdpd_list_rebuilds(tdpd_sys *s, int r, int64_t *out)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    if (r < 0 || r >= (int)s->reps.size() || !out) return fail(s, TDPD_EINVAL, "bad replica or output");
    uint32_t v = 0;
    if (s->use_list) {
        CU(cudaMemcpyAsync(&v, s->builds + r, sizeof v, cudaMemcpyDeviceToHost, exec_stream(s)));
        CU(cudaStreamSynchronize(exec_stream(s)));
    }
    *out = v;
    return TDPD_OK;
}

tdpd_status tdpd_step(tdpd_sys *s, int n)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    if (n < 0) return fail(s, TDPD_EINVAL, "negative step count");
    cudaStream_t st = exec_stream(s);
    int left = n;
    while (left >= GRAPH_LONG) {
        CU(cudaGraphLaunch(s->glong[s->parity], st));
        left -= GRAPH_LONG;
    }
    while (left > 0) {
        CU(cudaGraphLaunch(s->g1[s->parity], st));
        s->parity ^= 1;
        --left;
    }
    s->step += n;
    return TDPD_OK;
}

tdpd_status tdpd_step_timed(tdpd_sys *s, float *kernel_ms, int max_kernels, int *n_kernels)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    cudaStream_t st = exec_stream(s);
    CU(cudaGraphLaunch(s->gtimed[s->parity], st));
    CU(cudaStreamSynchronize(st));
    s->parity ^= 1;
    s->step += 1;
    const int nk = s->n_ev - 1;
    for (int k = 0; k < nk && k < max_kernels; ++k) CU(cudaEventElapsedTime(kernel_ms + k, s->ev[k], s->ev[k + 1]));
    if (n_kernels) *n_kernels = nk;
    return TDPD_OK;
}

const char *tdpd_kernel_name(const tdpd_sys *s, int k)
{
    if (!s) return nullptr;
    const std::vector<int> ks = step_kernels(s);
    return (k >= 0 && k < (int)ks.size()) ? KERNEL_NAMES[ks[k]] : nullptr;
}

tdpd_status tdpd_replica_status(tdpd_sys *s, int32_t *status)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    std::vector<uint32_t> w(s->reps.size());
    CU(cudaMemcpyAsync(w.data(), s->errw, sizeof(uint32_t) * w.size(), cudaMemcpyDeviceToHost, exec_stream(s)));
    CU(cudaStreamSynchronize(exec_stream(s)));
    for (size_t r = 0; r < w.size(); ++r)
        status[r] = (w[r] & 1u) ? TDPD_ENONFINITE : (w[r] & 2u) ? TDPD_EOVERFLOW : TDPD_OK;
    return TDPD_OK;
}

tdpd_status tdpd_sync(tdpd_sys *s)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    std::vector<int32_t> st(s->reps.size());
    if ((rc = tdpd_replica_status(s, st.data()))) return rc;
    for (size_t r = 0; r < st.size(); ++r)
        if (st[r] == TDPD_ENONFINITE) return fail(s, TDPD_ENONFINITE, "replica %zu produced a non-finite force", r);
        else if (st[r]) return fail(s, (tdpd_status)st[r], "replica %zu: a neighbour list overflowed", r);
    return TDPD_OK;
}

// ------------------------------------------------------------ checkpoint
// A checkpoint is the device state between two steps, byte for byte: the
// current buffer (sorted state, predicted values, forces and fluxes), the
// load-index map, the binning and list state, the step and membrane
// counters, the membranes' load-order predicted vertices, reference points,
// area/volume totals and constraint coefficients, and the status words. A
// handle committed with the same configuration continues from it exactly as
// the saved run would have (same slots, lists and random streams).

struct CkpHeader {
    char magic[8];
    uint32_t version;
    int32_t N, NC, ns, n_rep, n_rbc, lpp, use_list, nl_cap, parity, n_tiles;
    int64_t step;
    uint64_t cfg_hash;      // the device replica and membrane tables
    uint64_t nl_ints;       // list entries saved (list mode)
};

constexpr char CKP_MAGIC[8] = {'T', 'D', 'P', 'D', 'C', 'K', 'P', '1'};

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull)
{
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t k = 0; k < n; ++k) {
        h ^= c[k];
        h *= 1099511628211ull;
    }
    return h;
}

tdpd_status config_hash(tdpd_sys *s, uint64_t *out)
{
    std::vector<RepParams> P(s->reps.size());
    CU(cudaMemcpy(P.data(), s->d_reps, sizeof(RepParams) * P.size(), cudaMemcpyDeviceToHost));
    uint64_t h = fnv1a(P.data(), sizeof(RepParams) * P.size());
    if (s->n_rbc) {
        std::vector<RbcDev> R(s->n_rbc);
        CU(cudaMemcpy(R.data(), s->d_rbcs, sizeof(RbcDev) * R.size(), cudaMemcpyDeviceToHost));
        h = fnv1a(R.data(), sizeof(RbcDev) * R.size(), h);
    }
    *out = h;
    return TDPD_OK;
}

// (device pointer, bytes) of every saved array, in file order
std::vector<std::pair<void *, size_t>> ckp_arrays(tdpd_sys *s, int parity, size_t nl_ints)
{
    const size_t N = (size_t)s->N, ns = (size_t)s->ns, nr = s->reps.size(), nb = (size_t)s->n_rbc;
    const Buffers &B = s->buf[parity];
    std::vector<std::pair<void *, size_t>> v = {
        {B.pos, 16 * N}, {B.vt, 16 * N}, {B.vel, 16 * N}, {B.frc, 16 * N},
        {B.C, 4 * N * ns}, {B.Ct, 4 * N * ns}, {B.Q, 4 * N * ns},
        {s->inv, 4 * N}, {s->count, 4 * (size_t)s->n_tiles * SCAN_TILE},
        {s->tile_sum[0], 4 * (size_t)s->n_tiles}, {s->tile_sum[1], 4 * (size_t)s->n_tiles},
        {s->cellrank, 8 * N}, {s->errw, 4 * nr}, {s->step_ctr, 12}};
    if (s->use_list) {
        // the other buffer holds the next step's predicted state (written by
        // the pair epilogue), which a step without a rebuild uses as it is
        const Buffers &O = s->buf[1 - parity];
        v.push_back({O.pos, 16 * N});
        v.push_back({O.vt, 16 * N});
        v.push_back({O.vel, 16 * N});
        v.push_back({O.frc, 16 * N});
        v.push_back({O.C, 4 * N * ns});
        v.push_back({O.Ct, 4 * N * ns});
        v.push_back({O.Q, 4 * N * ns});
        v.push_back({s->disp[0], 4 * nr});
        v.push_back({s->disp[1], 4 * nr});
        v.push_back({s->builds, 4 * nr});
        v.push_back({s->nlc, 4 * N * (size_t)s->lpp});
        v.push_back({s->xb, 16 * N});
        v.push_back({s->nl, 4 * nl_ints});
    }
    if (nb) {
        v.push_back({s->mx, 16 * N});
        v.push_back({s->mv, 16 * N});
        for (int k = 0; k < 2; ++k) {
            v.push_back({s->d_ref[k], 16 * nb});
            v.push_back({s->d_av[k], 16 * nb});
            v.push_back({s->d_cgv[k], 8 * nb});
        }
    }
    return v;
}

size_t nl_used_ints(const tdpd_sys *s)
{
    return s->use_list ? ((size_t)s->N * s->lpp + 31) / 32 * 32 * (size_t)s->nl_cap : 0;
}

tdpd_status tdpd_save(tdpd_sys *s, const char *path)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    if (!path) return fail(s, TDPD_EINVAL, "null path");
    CkpHeader H{};
    std::memcpy(H.magic, CKP_MAGIC, 8);
    H.version = 2;     // 2: list mode also saves the other buffer
    H.N = s->N; H.NC = s->NC; H.ns = s->ns; H.n_rep = (int)s->reps.size(); H.n_rbc = s->n_rbc;
    H.lpp = s->lpp; H.use_list = s->use_list ? (s->half ? 2 : 1) : 0; H.nl_cap = s->nl_cap; H.parity = s->parity;
    H.n_tiles = s->n_tiles; H.step = s->step;
    H.nl_ints = nl_used_ints(s);
    CU(cudaStreamSynchronize(exec_stream(s)));
    if ((rc = config_hash(s, &H.cfg_hash))) return rc;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(s, TDPD_EINVAL, "cannot open %s for writing", path);
    bool ok = std::fwrite(&H, sizeof H, 1, f) == 1;
    std::vector<unsigned char> host;
    for (const auto &a : ckp_arrays(s, s->parity, H.nl_ints)) {
        if (!ok) break;
        host.resize(a.second);
        cudaError_t e = cudaMemcpy(host.data(), a.first, a.second, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            std::fclose(f);
            return fail(s, TDPD_ECUDA, "checkpoint read-back: %s", cudaGetErrorString(e));
        }
        ok = a.second == 0 || std::fwrite(host.data(), 1, a.second, f) == a.second;
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(s, TDPD_EINVAL, "writing %s failed", path);
    return TDPD_OK;
}

tdpd_status tdpd_load(tdpd_sys *s, const char *path)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    if (!path) return fail(s, TDPD_EINVAL, "null path");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(s, TDPD_EINVAL, "cannot open %s", path);
    CkpHeader H{};
    if (std::fread(&H, sizeof H, 1, f) != 1 || std::memcmp(H.magic, CKP_MAGIC, 8) != 0 || H.version != 2) {
        std::fclose(f);
        return fail(s, TDPD_EINVAL, "%s is not a checkpoint of this library", path);
    }
    uint64_t h = 0;
    if ((rc = config_hash(s, &h))) { std::fclose(f); return rc; }
    if (H.N != s->N || H.NC != s->NC || H.ns != s->ns || H.n_rep != (int)s->reps.size() || H.n_rbc != s->n_rbc ||
        (H.use_list != 0) != s->use_list || H.n_tiles != s->n_tiles || H.cfg_hash != h) {
        std::fclose(f);
        return fail(s, TDPD_EINVAL, "checkpoint of another configuration (particles, cells, species, replicas, "
                                    "membranes, list mode or parameters differ)");
    }
    if (H.lpp != s->lpp) {
        std::fclose(f);
        return fail(s, TDPD_EINVAL, "checkpoint taken with %d lanes per particle, this handle uses %d "
                                    "(tdpd_set_lanes before commit)", H.lpp, s->lpp);
    }
    if (s->use_list && H.use_list != (s->half ? 2 : 1)) {
        std::fclose(f);
        return fail(s, TDPD_EINVAL, "checkpoint taken with %s-shell lists, this handle uses %s-shell lists "
                                    "(tdpd_set_pair_mode before commit)", H.use_list == 2 ? "half" : "full",
                    s->half ? "half" : "full");
    }
    if (H.parity != 0 && H.parity != 1) {
        std::fclose(f);
        return fail(s, TDPD_EINVAL, "corrupt checkpoint header");
    }
    // the list layout follows the capacity of the saved run
    const bool recapture = s->use_list && H.nl_cap != s->nl_cap;
    if (s->use_list) {
        const size_t need = ((size_t)s->N * s->lpp + 31) / 32 * 32 * (size_t)H.nl_cap;
        if (H.nl_cap <= 0 || need != H.nl_ints) {
            std::fclose(f);
            return fail(s, TDPD_EINVAL, "corrupt checkpoint header");
        }
        if (need > s->nl_ints) {
            CU(cudaStreamSynchronize(exec_stream(s)));
            if (s->nl) CU(cudaFree(s->nl));
            s->nl = nullptr;
            s->nl_ints = 0;
            cudaError_t e = cudaMalloc(&s->nl, need * sizeof(int));
            if (e != cudaSuccess) {
                std::fclose(f);
                return fail(s, TDPD_ENOMEM, "neighbour lists (%zu bytes): %s", need * sizeof(int), cudaGetErrorString(e));
            }
            s->nl_ints = need;
        }
        s->nl_cap = H.nl_cap;
    }
    CU(cudaStreamSynchronize(exec_stream(s)));
    std::vector<unsigned char> host;
    bool ok = true;
    for (const auto &a : ckp_arrays(s, H.parity, H.nl_ints)) {
        host.resize(a.second);
        if (a.second && std::fread(host.data(), 1, a.second, f) != a.second) { ok = false; break; }
        cudaError_t e = cudaMemcpy(a.first, host.data(), a.second, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            std::fclose(f);
            return fail(s, TDPD_ECUDA, "checkpoint upload: %s", cudaGetErrorString(e));
        }
    }
    std::fclose(f);
    if (!ok) return fail(s, TDPD_EINVAL, "%s is truncated; the handle's state is undefined until the next load", path);
    s->parity = H.parity;
    s->step = H.step;
    if (recapture && (rc = capture_graphs(s))) return rc;
    return TDPD_OK;
}

tdpd_status tdpd_set_states_device(tdpd_sys *s, const float *pos, const float *vel, const float *conc)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    if (!pos || !vel || !conc) return fail(s, TDPD_EINVAL, "null array");
    const int N = s->N, ns = s->ns;
    cudaStream_t st = exec_stream(s);
    CU(cudaMemsetAsync(s->d_flag, 0, sizeof(uint32_t), st));
    launch_check_state(pos, vel, s->d_wstat, s->d_reps, N, s->d_flag, st);
    uint32_t bad = 0;
    CU(cudaMemcpyAsync(&bad, s->d_flag, sizeof bad, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (bad) return fail(s, TDPD_EINVAL, "a position outside its replica's box or a non-finite velocity");
    CU(cudaEventSynchronize(s->stage_done));
    CU(cudaMemcpyAsync(s->d_in, pos, sizeof(float) * 3 * (size_t)N, cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(s->d_in + 3 * (size_t)N, vel, sizeof(float) * 3 * (size_t)N, cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(s->d_in + 6 * (size_t)N, conc, sizeof(float) * (size_t)N * ns, cudaMemcpyDeviceToDevice, st));
    return init_device(s, false);
}

tdpd_status tdpd_read_state_device(tdpd_sys *s, int r, float *pos, float *vel, float *conc)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    HostRep *R = rep_of(s, r);
    if (!R) return fail(s, TDPD_EINVAL, "bad replica");
    launch_unpack_state(s->buf[s->parity], s->inv, s->rep_pbase[r], (int)R->type.size(), s->ns, pos, vel, conc,
                        s->d_flag, exec_stream(s));
    CU(cudaGetLastError());
    return TDPD_OK;
}

tdpd_status tdpd_set_states(tdpd_sys *s, const float *pos, const float *vel, const float *conc)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    if (!pos || !vel || !conc) return fail(s, TDPD_EINVAL, "null array");
    const int N = s->N, ns = s->ns;
    // the upload goes first (by DMA from pinned arrays); nothing is adopted
    // before the inputs pass the check. A large batch is checked on the
    // device (the host waits for one flag; a failed check is located on the
    // host, for the message); a small one on the host while the DMA runs,
    // which spares that round trip
    CU(cudaEventSynchronize(s->stage_done));
    cudaStream_t st = exec_stream(s);
    CU(cudaMemcpyAsync(s->d_in, pos, sizeof(float) * 3 * (size_t)N, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(s->d_in + 3 * (size_t)N, vel, sizeof(float) * 3 * (size_t)N, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(s->d_in + 6 * (size_t)N, conc, sizeof(float) * (size_t)N * ns, cudaMemcpyHostToDevice, st));
    bool bad = false;
    if (N > HOST_CHECK_MAX) {
        CU(cudaMemsetAsync(s->d_flag, 0, sizeof(uint32_t), st));
        launch_check_state(s->d_in, s->d_in + 3 * (size_t)N, s->d_wstat, s->d_reps, N, s->d_flag, st);
        uint32_t *flag = stage_ctr(s) + 3;
        CU(cudaMemcpyAsync(flag, s->d_flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        bad = *flag != 0u;
    }
    const long first = bad || N <= HOST_CHECK_MAX ? first_bad_particle(s, pos, vel) : -1;
    if (first >= 0 || bad) {
        CU(cudaStreamSynchronize(st));                // the caller's arrays are read
        const size_t r = first < 0 ? 0 : (size_t)(std::upper_bound(s->rep_pbase.begin(), s->rep_pbase.end(), (int)first) -
                                                  s->rep_pbase.begin()) - 1;
        return fail(s, TDPD_EINVAL, "replica %zu particle %ld: position outside the box or non-finite velocity", r,
                    first < 0 ? -1L : first - s->rep_pbase[r]);
    }
    if ((rc = init_device(s, false))) return rc;
    CU(cudaEventSynchronize(s->stage_done));         // the caller's arrays are read
    return TDPD_OK;
}

tdpd_status tdpd_set_state(tdpd_sys *s, int r, const float *pos, const float *vel, const float *conc)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    HostRep *R = rep_of(s, r);
    if (!R || !pos || !vel) return fail(s, TDPD_EINVAL, "bad replica or array");
    const int n = (int)R->type.size(), ns = s->ns;
    const float L0 = R->cfg.L[0], L1 = R->cfg.L[1], L2 = R->cfg.L[2];
    for (int i = 0; i < n; ++i) {
        const float *x = pos + 3 * (size_t)i, *v = vel + 3 * (size_t)i;
        const bool ok = x[0] >= 0.0f && x[0] < L0 && x[1] >= 0.0f && x[1] < L1 && x[2] >= 0.0f && x[2] < L2 &&
                        std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
        if (!ok) return fail(s, TDPD_EINVAL, "particle %d: position outside the box or non-finite velocity", i);
    }
    if (s->reps.size() == 1 && conc) {
        // one replica: the caller's arrays go to the device as they are (by DMA
        // when they are pinned) and are packed there; the host copy of the
        // state is left as it was, every other path refreshes it before use
        CU(cudaEventSynchronize(s->stage_done));
        cudaStream_t st = exec_stream(s);
        CU(cudaMemcpyAsync(s->d_in, pos, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(s->d_in + 3 * (size_t)n, vel, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(s->d_in + 6 * (size_t)n, conc, sizeof(float) * (size_t)n * ns, cudaMemcpyHostToDevice, st));
        if ((rc = init_device(s, false))) return rc;
        CU(cudaEventSynchronize(s->stage_done));     // the caller's arrays are read
        return TDPD_OK;
    }
    // other replicas keep their current device state
    for (size_t q = 0; q < s->reps.size(); ++q) {
        if ((int)q == r) continue;
        HostRep &O = s->reps[q];
        if ((rc = download(s, (int)q, O.pos.data(), O.vel.data(), O.conc.data(), nullptr, nullptr))) return rc;
    }
    if (!conc && (rc = download(s, r, nullptr, nullptr, R->conc.data(), nullptr, nullptr))) return rc;
    std::memcpy(R->pos.data(), pos, sizeof(float) * 3 * n);
    std::memcpy(R->vel.data(), vel, sizeof(float) * 3 * n);
    if (conc) std::memcpy(R->conc.data(), conc, sizeof(float) * (size_t)n * ns);
    return init_state(s);
}

tdpd_status tdpd_read_state(tdpd_sys *s, int r, float *pos, float *vel, float *conc)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    if (!rep_of(s, r)) return fail(s, TDPD_EINVAL, "bad replica");
    return download(s, r, pos, vel, conc, nullptr, nullptr);
}

tdpd_status tdpd_read_forces(tdpd_sys *s, int r, float *force, float *flux)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    if (!rep_of(s, r)) return fail(s, TDPD_EINVAL, "bad replica");
    return download(s, r, nullptr, nullptr, nullptr, force, flux);
}

tdpd_status tdpd_read_observables(tdpd_sys *s, int r, tdpd_obs *out)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    HostRep *R = rep_of(s, r);
    if (!R || !out) return fail(s, TDPD_EINVAL, "bad replica or output");
    cudaStream_t st = exec_stream(s);
    int c0 = -1, c1 = -1;
    for (size_t c = 0; c < s->h_chunks.size(); ++c)
        if (s->h_chunks[c].x == r) { if (c0 < 0) c0 = (int)c; c1 = (int)c + 1; }
    launch_observables(s->buf[s->parity], s->d_reps, s->d_chunks + c0, c1 - c0, s->ns, s->d_obs,
                       s->d_obs_tot, s->d_obs_done, st);
    CU(cudaMemcpyAsync(s->h_obs, s->d_obs_tot, sizeof(double) * OBS_K, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    const double *h = s->h_obs;
    std::memset(out, 0, sizeof *out);
    out->step = s->step + (s->reps.size() > 1 ? R->step : 0);
    out->n_particles = (int)R->type.size();
    out->n_species = s->ns;
    out->n_rbc = (int)R->rbcs.size();
    const double nm = h[4];
    out->n_mobile = (int)nm;
    for (int c = 0; c < 3; ++c) out->momentum[c] = h[c];
    const double p2 = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
    out->kT = nm > 1 ? (h[3] - p2 / nm) / (3.0 * (nm - 1.0)) : 0.0;
    out->n_membrane = (int)h[5];
    for (int k = 0; k < s->ns; ++k) {
        out->mass[k] = h[6 + k];
        out->mass_membrane[k] = h[6 + MAXS + k];
    }
    return TDPD_OK;
}

tdpd_status tdpd_read_rbc(tdpd_sys *s, int r, double *area, double *volume)
{
    tdpd_status rc = ensure(s);
    if (rc) return rc;
    HostRep *R = rep_of(s, r);
    if (!R) return fail(s, TDPD_EINVAL, "bad replica");
    const int nb = (int)R->rbcs.size();
    if (nb == 0) return TDPD_OK;
    std::vector<double2> av(nb);
    // the last K-Gather wrote the buffer of the last step's parity
    CU(cudaMemcpyAsync(av.data(), s->d_av[1 - s->parity] + s->rep_rbc0[r], sizeof(double2) * nb,
                       cudaMemcpyDeviceToHost, exec_stream(s)));
    CU(cudaStreamSynchronize(exec_stream(s)));
    for (int b = 0; b < nb; ++b) {
        if (area) area[b] = av[b].x;
        if (volume) volume[b] = av[b].y;
    }
    return TDPD_OK;
}

int tdpd_num_replicas(const tdpd_sys *s) { return s ? (int)s->reps.size() : 0; }

int tdpd_num_particles(const tdpd_sys *s, int r)
{
    if (!s || r < 0 || r >= (int)s->reps.size()) return -1;
    return (int)s->reps[r].type.size();
}

int64_t tdpd_current_step(const tdpd_sys *s) { return s ? s->step : -1; }

int tdpd_launches_per_step(const tdpd_sys *s)
{
    if (!s) return 0;
    // the half shell's pair entry is two launches (k_pair, k_pair_finish)
    return (int)step_kernels(s).size() + (s->committed && s->half ? 1 : 0);
}

const char *tdpd_last_error(const tdpd_sys *s) { return s ? s->err.c_str() : g_err.c_str(); }

void tdpd_destroy(tdpd_sys *s)
{
    if (!s) return;
    if (s->committed) cudaStreamSynchronize(exec_stream(s));
    free_device(s);
    if (s->own) cudaStreamDestroy(s->own);
    if (s->cap) cudaStreamDestroy(s->cap);
    delete s;
}

tdpd_status tdpd_debug_rng(uint64_t seed, int n, const uint32_t *i, const uint32_t *j,
                           const uint32_t *step, const uint32_t *stream, uint32_t *bits,
                           float *normal)
{
    tdpd_sys *s = nullptr;
    if (n < 0 || (n > 0 && (!i || !j || !step || !stream || !bits || !normal)))
        return fail(nullptr, TDPD_EINVAL, "bad arguments");
    if (n == 0) return TDPD_OK;
    uint32_t *d = nullptr;
    float *g = nullptr;
    const size_t sz = (size_t)n * sizeof(uint32_t);
    CU(cudaMalloc(&d, 6 * sz));
    cudaError_t e = cudaMalloc(&g, 2 * (size_t)n * sizeof(float));
    if (e != cudaSuccess) {
        cudaFree(d);
        return fail(nullptr, TDPD_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    cudaMemcpy(d, i, sz, cudaMemcpyHostToDevice);
    cudaMemcpy(d + n, j, sz, cudaMemcpyHostToDevice);
    cudaMemcpy(d + 2 * (size_t)n, step, sz, cudaMemcpyHostToDevice);
    cudaMemcpy(d + 3 * (size_t)n, stream, sz, cudaMemcpyHostToDevice);
    launch_debug_rng(seed, n, d, d + n, d + 2 * (size_t)n, d + 3 * (size_t)n, d + 4 * (size_t)n, g, 0);
    e = cudaMemcpy(bits, d + 4 * (size_t)n, 2 * sz, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(normal, g, 2 * (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(d);
    cudaFree(g);
    if (e != cudaSuccess) return fail(nullptr, TDPD_ECUDA, "debug rng: %s", cudaGetErrorString(e));
    return TDPD_OK;
}

}  // extern "C"
