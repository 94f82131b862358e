// tsim_api.cu -- C ABI of libtsim.so (declared in include/tsim.h): context
// lifetime, device memory, argument checks, the substep schedule (stream or
// CUDA graph with a device-driven relative-rest loop) and error latching.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tsim.h"
#include "tsim_device.cuh"
#include "tsim_kernels.h"

using namespace tsim;

static thread_local std::string g_err = "";

static int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(TSIM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

struct GraphChunk {
    int n = 0;
    cudaGraphExec_t exec = nullptr;
    // per substep three events: before the relative-rest loop, before the
    // commit transfer (= after the loop), after the commit transfer
    std::vector<cudaEvent_t> ev;
    bool pending = false;               // launched, timings not harvested
};

struct tsim_ctx {
    int n_inst = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    Dev d{};
    std::vector<Inst> hinst;
    std::vector<tsim_gel_desc> gels;
    std::vector<tsim_material> mats;
    tsim_solver_desc solver{};
    bool solver_set = false;
    std::vector<int> have_particles;
    std::vector<int> need_prologue;
    long long total_blocks = 0, total_nodes = 0, total_particles = 0, max_nodes = 0;
    long long total_objcap = 0;
    int max_nobj = 0;                   // most object particles of one instance (0: SDF contact everywhere)
    long long k_next = 0;
    int par_next = 0;
    // readout scratch
    float *ro = nullptr;                // num, den, height, normal (W*H*6 floats)
    int *ids = nullptr;                 // marker ids (4096)
    float *pick = nullptr;              // marker positions (4096*3)
    // graph execution
    bool use_graph = false;
    std::vector<GraphChunk> chunks;     // ring of graph executables of chunk_len substeps
    int chunk_next = 0;
    // execution configuration (tsim_set_tuning / tsim_autotune); no effect on results
    int chunk_len = 20;
    int grid_threads = 256, grid_flat = 0;
    float tuned_us = 0.f;
    // profiling of the commit transfer
    bool profile = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    long long prof_launches = 0;
    double prof_ms = 0.0;
    double prof_loop_ms = 0.0;          // time inside the relative-rest loops (repeat passes)
};

static const int RO_MAX = 1 << 20;
static const int MARK_MAX = 4096;

extern "C" const char *tsim_last_error(void) { return g_err.c_str(); }

extern "C" int tsim_block_slots(void) { return block_slots(); }

// used by the allocation-free entry point (tsim_noalloc.cu) to report through tsim_last_error
void tsim_record_error(const std::string &msg) { g_err = msg; }

static void free_all(tsim_ctx *c)
{
    Dev &d = c->d;
    void *ptrs[] = {d.P[0], d.P[1], d.T[0], d.T[1], d.cnt[0], d.cnt[1], d.VC, d.acc, d.vel, d.sortc, d.objq,
                    d.blk_inst, d.inst, d.ist, d.G, (void *)d.kf, (void *)d.perm, d.log,
                    d.sx, d.sv, d.sC, d.sF, d.stag, c->ro, c->ids, c->pick, (void *)d.gchunk};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &g : c->chunks) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        for (auto e : g.ev) cudaEventDestroy(e);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    d = Dev{};
}

static void fill_material(Inst &I, const tsim_gel_desc &g, const tsim_material &m, float dt)
{
    double dx = g.dx;
    double V0 = dx * dx * dx / g.ppc;
    I.dx = g.dx;
    I.inv_dx = (float)(1.0 / dx);
    I.V0 = (float)V0;
    I.mp = (float)(m.rho * V0);
    I.mu = (float)(m.E / (2.0 * (1.0 + m.nu)));
    I.lam = (float)(m.E * m.nu / ((1.0 + m.nu) * (1.0 - 2.0 * m.nu)));
    I.dt = dt;
    I.kME = (float)(-4.0 * dt * V0 / (dx * dx));
    for (int a = 0; a < 3; ++a) I.g[a] = m.gravity[a];
}

static int upload_inst(tsim_ctx *c)
{
    CU(cudaMemcpyAsync(c->d.inst, c->hinst.data(), sizeof(Inst) * c->n_inst, cudaMemcpyHostToDevice,
                       c->stream));
    return TSIM_OK;
}

static int check_ctx(tsim_ctx *c, int inst)
{
    if (!c) return fail(TSIM_ERR_INVALID_ARG, "null context");
    if (inst < 0 || inst >= c->n_inst) return fail(TSIM_ERR_INVALID_ARG, "instance index out of range");
    return TSIM_OK;
}

extern "C" int tsim_create(int n_inst, const tsim_gel_desc *gels, const tsim_material *mats,
                           void *stream, tsim_ctx **out)
{
    if (!out) return fail(TSIM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_inst < 1 || n_inst > 65535 || !gels || !mats)
        return fail(TSIM_ERR_INVALID_ARG, "need 1..65535 instances and descriptor arrays");
    tsim_ctx *c = new tsim_ctx();
    c->n_inst = n_inst;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    c->hinst.resize(n_inst);
    c->gels.assign(gels, gels + n_inst);
    c->mats.assign(mats, mats + n_inst);
    c->have_particles.assign(n_inst, 0);
    c->need_prologue.assign(n_inst, 0);
    long long blocks = 0, nodes = 0, parts = 0;
    for (int i = 0; i < n_inst; ++i) {
        const tsim_gel_desc &g = gels[i];
        const tsim_material &m = mats[i];
        bool ok = g.cx > 0 && g.cy > 0 && g.cz > 0 && g.ppc == 8 && g.dx > 0.f && std::isfinite(g.dx) &&
                  g.nx % BLK == 0 && g.ny % BLK == 0 && g.nz % BLK == 0 && g.ox >= 2 && g.oy >= 2 &&
                  g.oz >= 2 && g.ox + g.cx + 2 <= g.nx && g.oy + g.cy + 2 <= g.ny && g.oz + g.cz + 2 <= g.nz &&
                  m.E > 0.f && m.nu >= 0.f && m.nu < 0.5f && m.rho > 0.f &&
                  (long long)g.nx * g.ny * g.nz < (1ll << 31);
        long long np = (long long)g.cx * g.cy * g.cz * g.ppc;
        if (!ok || np > (long long)ID_MASK) {
            delete c;
            return fail(TSIM_ERR_INVALID_ARG, "instance " + std::to_string(i) +
                                                  ": bad gel or material descriptor (node box must be a "
                                                  "multiple of 4, below 2^31 nodes, and hold the gel "
                                                  "with a 2-node margin; ppc must be 8; 0 <= nu < 0.5)");
        }
        Inst &I = c->hinst[i];
        memset(&I, 0, sizeof(Inst));
        I.nx = g.nx; I.ny = g.ny; I.nz = g.nz;
        I.ox = g.ox; I.oy = g.oy; I.oz = g.oz;
        I.nbx = g.nx / BLK; I.nby = g.ny / BLK; I.nbz = g.nz / BLK;
        I.nblocks = I.nbx * I.nby * I.nbz;
        I.block0 = (int)blocks;
        I.n_particles = (int)np;
        I.node0 = nodes;
        I.id0 = parts;
        I.H = g.cz * g.dx;
        I.limit = 1;
        I.threshold = 0.5f;
        I.ind_kind = K_NONE;
        I.walls = 1;
        fill_material(I, g, m, 1e-5f);
        I.spc = (int)std::max(4096ll, (np / 16 + 3) / 4 * 4);
        I.objcap = (int)std::max(65536ll, np / 4);
        I.obj0 = c->total_objcap;
        c->total_objcap += I.objcap;
        blocks += I.nblocks;
        long long nn = (long long)g.nx * g.ny * g.nz;
        nodes += nn;
        if (nn > c->max_nodes) c->max_nodes = nn;
        parts += np;
    }
    long long spill = 0;
    for (int i = 0; i < n_inst; ++i) {              // spill slots follow the cell blocks' slots
        c->hinst[i].sp0 = blocks * (long long)CAP + spill;
        spill += c->hinst[i].spc;
    }
    if (blocks * (long long)CAP + spill > (1ll << 31) || blocks > (1ll << 30)) {
        delete c;
        return fail(TSIM_ERR_INVALID_ARG, "problem too large");
    }
    {
        cudaError_t e = setup_kernels();
        if (e != cudaSuccess) {
            delete c;
            return fail(TSIM_ERR_CUDA, std::string("kernel setup: ") + cudaGetErrorString(e));
        }
    }
    c->total_blocks = blocks;
    c->total_nodes = nodes;
    c->total_particles = parts;
    Dev &d = c->d;
    // packed grid-update launch table: 128-node chunks, instances padded to 512 nodes
    std::vector<int2> gch;
    for (int i = 0; i < n_inst; ++i) {
        const long long nn = (long long)c->hinst[i].nx * c->hinst[i].ny * c->hinst[i].nz;
        const long long nch = (nn + 511) / 512 * 4, first = (long long)gch.size();
        for (long long a = 0; a < nch; ++a) gch.push_back(make_int2(i, (int)first));
    }
    d.n_gchunk = (long long)gch.size();
    d.S = blocks * CAP + spill;
    d.n_inst = n_inst;
    d.n_blocks = (int)blocks;
    const size_t S = (size_t)d.S;
    struct A {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&d.P[0], S * 12 * sizeof(float)},      {(void **)&d.P[1], S * 12 * sizeof(float)},
        {(void **)&d.T[0], S * sizeof(uint32_t)},         {(void **)&d.T[1], S * sizeof(uint32_t)},
        {(void **)&d.cnt[0], blocks * sizeof(int)},       {(void **)&d.cnt[1], blocks * sizeof(int)},
        {(void **)&d.VC, S * 12 * sizeof(float)},         {(void **)&d.acc, nodes * sizeof(float4)},
        {(void **)&d.vel, nodes * sizeof(float4)},
        {(void **)&d.blk_inst, blocks * sizeof(int)},     {(void **)&d.sortc, blocks * SORTC * sizeof(unsigned short)},
        {(void **)&d.objq, (size_t)c->total_objcap * sizeof(float4)},     {(void **)&d.inst, n_inst * sizeof(Inst)},
        {(void **)&d.ist, n_inst * sizeof(InstState)},    {(void **)&d.G, sizeof(Global)},
        {(void **)&d.kf, n_inst * MAX_KF * 5 * sizeof(float)},
        {(void **)&d.perm, n_inst * 256 * sizeof(int)},   {(void **)&d.log, n_inst * LOGN * sizeof(int2)},
        {(void **)&d.sx, parts * 3 * sizeof(float)},      {(void **)&d.sv, parts * 3 * sizeof(float)},
        {(void **)&d.sC, parts * 9 * sizeof(float)},      {(void **)&d.sF, parts * 9 * sizeof(float)},
        {(void **)&d.stag, parts * sizeof(uint32_t)},     {(void **)&c->ro, (size_t)RO_MAX * 6 * sizeof(float)},
        {(void **)&c->ids, MARK_MAX * sizeof(int)},       {(void **)&c->pick, MARK_MAX * 3 * sizeof(float)},
        {(void **)&d.gchunk, gch.size() * sizeof(int2)},
    };
    for (auto &a : allocs) {
        cudaError_t e = cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_all(c);
            delete c;
            return fail(TSIM_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(a.bytes) +
                                          " bytes failed: " + cudaGetErrorString(e));
        }
    }
    std::vector<int> bi(blocks);
    for (int i = 0; i < n_inst; ++i)
        for (int b = 0; b < c->hinst[i].nblocks; ++b) bi[c->hinst[i].block0 + b] = i;
    int rc = TSIM_OK;
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == TSIM_OK) rc = fail(TSIM_ERR_CUDA, cudaGetErrorString(e));
    };
    chk(cudaMemsetAsync(d.cnt[0], 0, blocks * sizeof(int), c->stream));
    chk(cudaMemsetAsync(d.cnt[1], 0, blocks * sizeof(int), c->stream));
    chk(cudaMemsetAsync(d.acc, 0, nodes * sizeof(float4), c->stream));
    chk(cudaMemsetAsync(d.vel, 0, nodes * sizeof(float4), c->stream));
    chk(cudaMemsetAsync(d.ist, 0, n_inst * sizeof(InstState), c->stream));
    chk(cudaMemsetAsync(d.G, 0, sizeof(Global), c->stream));
    chk(cudaMemsetAsync((void *)d.kf, 0, n_inst * MAX_KF * 5 * sizeof(float), c->stream));
    chk(cudaMemsetAsync(d.log, 0, n_inst * LOGN * sizeof(int2), c->stream));
    chk(cudaMemsetAsync(d.VC, 0, S * 12 * sizeof(float), c->stream));
    chk(cudaMemsetAsync(d.sortc, 0, blocks * SORTC * sizeof(unsigned short), c->stream));
    chk(cudaMemcpyAsync(d.blk_inst, bi.data(), blocks * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    chk(cudaMemcpyAsync((void *)d.gchunk, gch.data(), gch.size() * sizeof(int2), cudaMemcpyHostToDevice,
                        c->stream));
    std::vector<int> perm(n_inst * 256);
    for (int i = 0; i < n_inst; ++i)
        for (int a = 0; a < 256; ++a) perm[i * 256 + a] = a;
    chk(cudaMemcpyAsync((void *)d.perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice,
                        c->stream));
    if (rc == TSIM_OK) rc = upload_inst(c);
    if (rc == TSIM_OK) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = fail(TSIM_ERR_CUDA, cudaGetErrorString(e));
    }
    if (rc != TSIM_OK) {
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return TSIM_OK;
}

extern "C" void tsim_destroy(tsim_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

static void invalidate_graphs(tsim_ctx *c)
{
    for (auto &g : c->chunks) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        for (auto e : g.ev) cudaEventDestroy(e);
    }
    c->chunks.clear();
}

static void mark_all_prologue(tsim_ctx *c)
{
    for (int i = 0; i < c->n_inst; ++i)
        if (c->have_particles[i]) c->need_prologue[i] = 1;
}

extern "C" int tsim_set_solver(tsim_ctx *c, const tsim_solver_desc *s)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    if (!s || !(s->dt > 0.f) || !std::isfinite(s->dt) || s->relrest_limit < 1 || s->relrest_limit > 1000 ||
        !(s->relrest_threshold >= 0.f) || s->base_mode < 0 || s->base_mode > 2)
        return fail(TSIM_ERR_INVALID_ARG, "bad solver descriptor (dt > 0, 1 <= limit <= 1000, threshold >= 0)");
    c->solver = *s;
    c->solver_set = true;
    for (int i = 0; i < c->n_inst; ++i) {
        Inst &I = c->hinst[i];
        fill_material(I, c->gels[i], c->mats[i], s->dt);
        I.limit = s->relrest_limit;
        I.threshold = s->relrest_threshold;
        I.base_mode = s->base_mode;
        I.walls = s->walls ? 1 : 0;
    }
    invalidate_graphs(c);
    mark_all_prologue(c);
    return upload_inst(c);
}

extern "C" int tsim_set_indenter(tsim_ctx *c, int inst, const tsim_indenter_desc *ind)
{
    int rc = check_ctx(c, inst);
    if (rc) return rc;
    if (!ind || ind->kind < -1 || ind->kind > 4 || !(ind->mu >= 0.f) || !std::isfinite(ind->mu_kinetic) ||
        ind->mu_kinetic > ind->mu)
        return fail(TSIM_ERR_INVALID_ARG, "bad indenter descriptor (mu >= 0, mu_kinetic <= mu)");
    for (int a = 0; a < 8; ++a)
        if (!std::isfinite(ind->p[a])) return fail(TSIM_ERR_INVALID_ARG, "non-finite indenter parameter");
    if (ind->kind == TSIM_PERLIN) {
        if (!(ind->p[5] > 0.f) || ind->p[7] < 0.f || ind->p[7] > 16.f)
            return fail(TSIM_ERR_INVALID_ARG, "Perlin plate needs period > 0 and 0..16 octaves");
        for (int a = 0; a < 256; ++a)
            if (ind->perm[a] < 0 || ind->perm[a] > 255)
                return fail(TSIM_ERR_INVALID_ARG, "permutation entries must be 0..255");
    }
    Inst &I = c->hinst[inst];
    I.ind_kind = ind->kind;
    for (int a = 0; a < 8; ++a) I.ip[a] = ind->p[a];
    I.fric = ind->mu;
    I.fric_k = ind->mu_kinetic > 0.f ? ind->mu_kinetic : ind->mu;
    I.tip_offset = ind->tip_offset;
    CU(cudaMemcpyAsync((void *)(c->d.perm + inst * 256), ind->perm, 256 * sizeof(int), cudaMemcpyHostToDevice,
                       c->stream));
    if (c->have_particles[inst]) c->need_prologue[inst] = 1;
    return upload_inst(c);
}

extern "C" int tsim_set_object_particles(tsim_ctx *c, int inst, const float *q, int n, float mass, int on_device)
{
    int rc = check_ctx(c, inst);
    if (rc) return rc;
    Inst &I = c->hinst[inst];
    if (n < 0 || n > I.objcap || (n > 0 && (!q || !(mass > 0.f) || !std::isfinite(mass))))
        return fail(TSIM_ERR_INVALID_ARG, "object particles: 0 <= n <= " + std::to_string(I.objcap) +
                                              ", positions given and mass > 0");
    if (n > 0) {
        // xyz rows of 12 bytes into float4 slots of 16
        CU(cudaMemcpy2DAsync(c->d.objq + I.obj0, sizeof(float4), q, 3 * sizeof(float), 3 * sizeof(float), (size_t)n,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    }
    I.nobj = n;
    I.objm = n > 0 ? mass : 0.f;
    int mx = 0;
    for (int i = 0; i < c->n_inst; ++i) mx = std::max(mx, c->hinst[i].nobj);
    if ((mx > 0) != (c->max_nobj > 0) || mx > c->max_nobj) invalidate_graphs(c);
    c->max_nobj = mx;
    if (c->have_particles[inst]) c->need_prologue[inst] = 1;
    rc = upload_inst(c);
    if (rc) return rc;
    CU(cudaStreamSynchronize(c->stream));      // host arrays may be freed after return
    return TSIM_OK;
}

extern "C" int tsim_set_trajectory(tsim_ctx *c, int inst, const tsim_keyframe *kf, int n_kf, int on_device)
{
    int rc = check_ctx(c, inst);
    if (rc) return rc;
    if (!kf || n_kf < 1 || n_kf > MAX_KF) return fail(TSIM_ERR_INVALID_ARG, "need 1..64 keyframes");
    std::vector<tsim_keyframe> h(n_kf);
    if (on_device) {
        CU(cudaMemcpyAsync(h.data(), kf, sizeof(tsim_keyframe) * n_kf, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    } else {
        memcpy(h.data(), kf, sizeof(tsim_keyframe) * n_kf);
    }
    std::vector<float> rows(MAX_KF * 5, 0.f);
    for (int a = 0; a < n_kf; ++a) {
        if (a > 0 && h[a].substep <= h[a - 1].substep)
            return fail(TSIM_ERR_INVALID_ARG, "keyframe substeps must increase");
        if (h[a].substep < 0 || h[a].substep > (1 << 24))
            return fail(TSIM_ERR_INVALID_ARG, "keyframe substep out of range");
        rows[a * 5] = (float)h[a].substep;
        for (int d = 0; d < 3; ++d) rows[a * 5 + 1 + d] = h[a].tip[d];
        rows[a * 5 + 4] = h[a].yaw;
        for (int d = 1; d < 5; ++d)
            if (!std::isfinite(rows[a * 5 + d])) return fail(TSIM_ERR_INVALID_ARG, "non-finite keyframe");
    }
    // the host copy lives until the copy ran: copy synchronously from pageable memory
    CU(cudaMemcpyAsync((void *)(c->d.kf + (size_t)inst * MAX_KF * 5), rows.data(), rows.size() * sizeof(float),
                       cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->hinst[inst].nkf = n_kf;
    if (c->have_particles[inst]) c->need_prologue[inst] = 1;
    return upload_inst(c);
}

extern "C" int tsim_set_substep(tsim_ctx *c, int64_t k)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    if (k < 0) return fail(TSIM_ERR_INVALID_ARG, "substep must be >= 0");
    c->k_next = k;
    long long kk = k;
    CU(cudaMemcpyAsync(&c->d.G->k_next, &kk, sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    mark_all_prologue(c);
    return TSIM_OK;
}

static int latched(tsim_ctx *c);

static int set_dirty(tsim_ctx *c, int inst, int v)
{
    CU(cudaMemcpyAsync(&c->d.ist[inst].dirty, &v, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));   // v lives on this frame
    return TSIM_OK;
}

// P2G of the stored state (x, F in slots, v and C in VC) for one instance.
static int run_prologue(tsim_ctx *c, int inst)
{
    const Inst &I = c->hinst[inst];
    CU(cudaMemsetAsync(c->d.acc + I.node0, 0, sizeof(float4) * (size_t)I.nx * I.ny * I.nz, c->stream));
    CU(cudaMemsetAsync(&c->d.ist[inst].e_key, 0xff, sizeof(unsigned long long), c->stream));
    int rc = set_dirty(c, inst, 1);
    if (rc) return rc;
    launch_transfer(c->d, MODE_PROLOGUE_, I.block0, I.nblocks, c->stream);
    launch_object_p2g(c->d, MODE_PROLOGUE_, inst, 1, I.nobj, c->stream);
    CU(cudaGetLastError());
    rc = set_dirty(c, inst, 0);
    if (rc) return rc;
    c->need_prologue[inst] = 0;
    return TSIM_OK;
}

static int pending_prologues(tsim_ctx *c)
{
    for (int i = 0; i < c->n_inst; ++i)
        if (c->need_prologue[i]) {
            int rc = run_prologue(c, i);
            if (rc) return rc;
        }
    return TSIM_OK;
}

extern "C" int tsim_write_particles(tsim_ctx *c, int inst, const float *x, const float *v, const float *C,
                                    const float *F, const uint32_t *tag, int n, int on_device)
{
    int rc = check_ctx(c, inst);
    if (rc) return rc;
    if (!c->solver_set) return fail(TSIM_ERR_STATE, "tsim_set_solver must precede tsim_write_particles");
    const Inst &I = c->hinst[inst];
    if (n != I.n_particles) return fail(TSIM_ERR_INVALID_ARG, "n must equal cx*cy*cz*ppc");
    if (!x || !v || !C || !F || !tag) return fail(TSIM_ERR_INVALID_ARG, "null particle array");
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const Dev &d = c->d;
    const size_t o = (size_t)I.id0;
    CU(cudaMemcpyAsync(d.sx + o * 3, x, sizeof(float) * 3 * n, kind, c->stream));
    CU(cudaMemcpyAsync(d.sv + o * 3, v, sizeof(float) * 3 * n, kind, c->stream));
    CU(cudaMemcpyAsync(d.sC + o * 9, C, sizeof(float) * 9 * n, kind, c->stream));
    CU(cudaMemcpyAsync(d.sF + o * 9, F, sizeof(float) * 9 * n, kind, c->stream));
    CU(cudaMemcpyAsync(d.stag + o, tag, sizeof(uint32_t) * n, kind, c->stream));
    CU(cudaMemsetAsync(d.cnt[c->par_next] + I.block0, 0, sizeof(int) * I.nblocks, c->stream));
    CU(cudaMemsetAsync(&d.ist[inst].nsp[c->par_next], 0, sizeof(int), c->stream));
    launch_bin_staged(d, inst, n, c->par_next, c->stream);
    CU(cudaGetLastError());
    c->have_particles[inst] = 1;
    rc = run_prologue(c, inst);
    if (rc) return rc;
    return latched(c);                      // synchronises: host arrays may be freed after return
}

// ---------------------------------------------------------------- substep schedule

static int launch_substeps_stream(tsim_ctx *c, int n)
{
    const int limit = c->solver.relrest_limit;
    for (int s = 0; s < n; ++s) {
        launch_round_begin(c->d, c->stream);
        launch_grid(c->d, c->max_nodes, c->grid_threads, c->grid_flat, c->stream);   // with the check
        cudaEvent_t ew = nullptr, e0 = nullptr, e1 = nullptr;
        if (c->profile) {
            if (c->ev_used + 3 > c->ev_pool.size()) {
                for (int a = 0; a < 255; ++a) {
                    cudaEvent_t e;
                    CU(cudaEventCreate(&e));
                    c->ev_pool.push_back(e);
                }
            }
            ew = c->ev_pool[c->ev_used++];
            e0 = c->ev_pool[c->ev_used++];
            e1 = c->ev_pool[c->ev_used++];
            CU(cudaEventRecord(ew, c->stream));
        }
        for (int j = 1; j < limit; ++j) {
            launch_transfer(c->d, MODE_ITER_, 0, (int)c->total_blocks, c->stream);
            launch_object_p2g(c->d, MODE_ITER_, 0, c->n_inst, c->max_nobj, c->stream);
            launch_grid(c->d, c->max_nodes, c->grid_threads, c->grid_flat, c->stream);
        }
        if (c->profile) CU(cudaEventRecord(e0, c->stream));
        launch_transfer(c->d, MODE_COMMIT_, 0, (int)c->total_blocks, c->stream);
        launch_object_p2g(c->d, MODE_COMMIT_, 0, c->n_inst, c->max_nobj, c->stream);
        if (c->profile) CU(cudaEventRecord(e1, c->stream));
        CU(cudaGetLastError());
    }
    return TSIM_OK;
}

static int add_kernel(cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *deps, int ndeps, void *fn,
                      dim3 grid, dim3 block, void **args, size_t shmem = 0)
{
    cudaKernelNodeParams p{};
    p.func = fn;
    p.gridDim = grid;
    p.blockDim = block;
    p.sharedMemBytes = (unsigned int)shmem;
    p.kernelParams = args;
    p.extra = nullptr;
    CU(cudaGraphAddKernelNode(node, g, deps, ndeps, &p));
    return TSIM_OK;
}

// Graph of n substeps: R0 -> grid+check -> WHILE{ transfer(ITER) -> grid+check }
// -> [event] -> transfer(COMMIT) -> [event], chained n times (the relative-rest
// check runs in CTA 0 of every grid update launch).
static int build_chunk(tsim_ctx *c, int n, GraphChunk &out)
{
    cudaGraph_t g;
    CU(cudaGraphCreate(&g, 0));
    int rc = TSIM_OK;
    Dev d = c->d;
    int zero = 0;
    dim3 grid_grid, grid_blk;
    grid_launch_shape(d, c->max_nodes, c->grid_threads, c->grid_flat, grid_grid, grid_blk);
    const dim3 tr_grid((unsigned int)c->total_blocks), tr_blk(NT), sp_grid(SPILL_CTAS);
    const dim3 obj_grid((unsigned int)((c->max_nobj + 255) / 256), (unsigned int)c->n_inst);
    cudaGraphNode_t prev = nullptr;
    out.n = n;
    for (auto e : out.ev) cudaEventDestroy(e);
    out.ev.clear();
    for (int s = 0; s < n && rc == TSIM_OK; ++s) {
        cudaGraphConditionalHandle h;
        CU(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
        int use1 = 1;
        void *a_r0[] = {&d};
        void *a_spill[] = {&d};
        void *a_grid[] = {&d, &h, &use1};
        void *a_tr[] = {&d, &zero};
        void *a_obj[] = {&d, &zero};
        cudaGraphNode_t n_r0, n_chk, n_while, n_ev0 = nullptr, n_commit, n_ev1;
        rc = add_kernel(g, &n_r0, prev ? &prev : nullptr, prev ? 1 : 0, fn_round_begin(),
                        dim3(round_begin_ctas(d)), dim3(256), a_r0);
        if (rc) break;
        rc = add_kernel(g, &n_chk, &n_r0, 1, fn_grid(c->grid_flat), grid_grid, grid_blk, a_grid);
        if (rc) break;
        cudaGraphNodeParams wp{};
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = h;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        // with profiling an event before the loop node (event nodes cannot sit
        // inside a conditional body, so the loop is timed whole)
        cudaGraphNode_t while_deps[2] = {n_chk, nullptr};
        int n_while_deps = 1;
        cudaEvent_t ew = nullptr, e0 = nullptr, e1 = nullptr;
        if (c->profile) {
            CU(cudaEventCreate(&ew));
            CU(cudaEventCreate(&e0));
            CU(cudaEventCreate(&e1));
            out.ev.push_back(ew);
            out.ev.push_back(e0);
            out.ev.push_back(e1);
            CU(cudaGraphAddEventRecordNode(&while_deps[1], g, &n_chk, 1, ew));
            n_while_deps = 2;
        }
        CU(cudaGraphAddNode(&n_while, g, while_deps, nullptr, n_while_deps, &wp));
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        cudaGraphNode_t b_tr[3], b_chk;
        int n_tr = 2;
        // the transfer of the cell blocks and of the spill slots run side by side
        rc = add_kernel(body, &b_tr[0], nullptr, 0, fn_transfer(MODE_ITER_), tr_grid, tr_blk, a_tr,
                        transfer_smem_bytes());
        if (rc) break;
        rc = add_kernel(body, &b_tr[1], nullptr, 0, fn_spill(MODE_ITER_), sp_grid, tr_blk, a_spill);
        if (rc) break;
        if (c->max_nobj > 0) {           // the particle-represented indenter, a third parallel branch
            rc = add_kernel(body, &b_tr[2], nullptr, 0, fn_object_p2g(MODE_ITER_), obj_grid, dim3(256), a_obj);
            if (rc) break;
            n_tr = 3;
        }
        rc = add_kernel(body, &b_chk, b_tr, n_tr, fn_grid(c->grid_flat), grid_grid, grid_blk, a_grid);
        if (rc) break;
        cudaGraphNode_t last = n_while;
        if (c->profile) {
            CU(cudaGraphAddEventRecordNode(&n_ev0, g, &last, 1, e0));
            last = n_ev0;
        }
        cudaGraphNode_t n_commits[3];
        int n_cm = 2;
        rc = add_kernel(g, &n_commits[0], &last, 1, fn_transfer(MODE_COMMIT_), tr_grid, tr_blk, a_tr,
                        transfer_smem_bytes());
        if (rc) break;
        rc = add_kernel(g, &n_commits[1], &last, 1, fn_spill(MODE_COMMIT_), sp_grid, tr_blk, a_spill);
        if (rc) break;
        if (c->max_nobj > 0) {
            rc = add_kernel(g, &n_commits[2], &last, 1, fn_object_p2g(MODE_COMMIT_), obj_grid, dim3(256), a_obj);
            if (rc) break;
            n_cm = 3;
        }
        if (c->profile) {
            CU(cudaGraphAddEventRecordNode(&n_ev1, g, n_commits, n_cm, out.ev.back()));
            prev = n_ev1;
        } else {
            CU(cudaGraphAddEmptyNode(&n_commit, g, n_commits, n_cm));
            prev = n_commit;
        }
    }
    if (rc == TSIM_OK) {
        cudaError_t e = cudaGraphInstantiate(&out.exec, g, 0);
        if (e != cudaSuccess) rc = fail(TSIM_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    cudaGraphDestroy(g);
    return rc;
}

// events in triples (loop start, commit start, commit end) per substep
static int harvest_events(tsim_ctx *c, const std::vector<cudaEvent_t> &ev, size_t n)
{
    for (size_t a = 0; a + 3 <= n; a += 3) {
        CU(cudaEventSynchronize(ev[a + 2]));
        float ms = 0.f, lms = 0.f;
        CU(cudaEventElapsedTime(&lms, ev[a], ev[a + 1]));
        CU(cudaEventElapsedTime(&ms, ev[a + 1], ev[a + 2]));
        c->prof_ms += ms;
        c->prof_loop_ms += lms;
        c->prof_launches += 1;
    }
    return TSIM_OK;
}

static int harvest(tsim_ctx *c, GraphChunk &g)
{
    if (!g.pending) return TSIM_OK;
    int rc = harvest_events(c, g.ev, g.ev.size());
    if (rc) return rc;
    g.pending = false;
    return TSIM_OK;
}

static int harvest_stream(tsim_ctx *c)
{
    int rc = harvest_events(c, c->ev_pool, c->ev_used);
    if (rc) return rc;
    c->ev_used = 0;
    return TSIM_OK;
}

static int ensure_chunks(tsim_ctx *c)
{
    if (!c->chunks.empty()) return TSIM_OK;
    c->chunks.resize(3);
    for (int a = 0; a < 2; ++a) {
        int rc = build_chunk(c, c->chunk_len, c->chunks[a]);
        if (rc) return rc;
    }
    c->chunks[2].n = 0;
    c->chunk_next = 0;
    return TSIM_OK;
}

static int launch_substeps_graph(tsim_ctx *c, int n)
{
    int rc = ensure_chunks(c);
    if (rc) return rc;
    const int L = c->chunk_len;
    int left = n;
    while (left >= L) {
        GraphChunk &g = c->chunks[c->chunk_next];
        rc = harvest(c, g);
        if (rc) return rc;
        CU(cudaGraphLaunch(g.exec, c->stream));
        g.pending = c->profile;
        c->chunk_next ^= 1;
        left -= L;
    }
    if (left > 0) {
        GraphChunk &g = c->chunks[2];
        rc = harvest(c, g);
        if (rc) return rc;
        if (g.n != left || !g.exec) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            rc = build_chunk(c, left, g);
            if (rc) return rc;
        }
        CU(cudaGraphLaunch(g.exec, c->stream));
        g.pending = c->profile;
    }
    return TSIM_OK;
}

static int check_steppable(tsim_ctx *c)
{
    for (int i = 0; i < c->n_inst; ++i)
        if (!c->have_particles[i])
            return fail(TSIM_ERR_STATE, "instance " + std::to_string(i) + " has no particles");
    return pending_prologues(c);
}

// n >= 1 substeps with the current execution configuration
static int step_n(tsim_ctx *c, int n)
{
    launch_set_end(c->d, n, c->stream);
    CU(cudaGetLastError());
    int rc = c->use_graph ? launch_substeps_graph(c, n) : launch_substeps_stream(c, n);
    if (rc) return rc;
    c->k_next += n;
    c->par_next ^= (n & 1);
    return TSIM_OK;
}

extern "C" int tsim_step(tsim_ctx *c, int n)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    if (n < 0) return fail(TSIM_ERR_INVALID_ARG, "n_substeps must be >= 0");
    if (n == 0) return TSIM_OK;
    rc = check_steppable(c);
    if (rc) return rc;
    return step_n(c, n);
}

static int latched(tsim_ctx *c)
{
    CU(cudaStreamSynchronize(c->stream));
    std::vector<InstState> h(c->n_inst);
    CU(cudaMemcpy(h.data(), c->d.ist, sizeof(InstState) * c->n_inst, cudaMemcpyDeviceToHost));
    unsigned int st = 0;
    int first = -1;
    for (int i = 0; i < c->n_inst; ++i) {
        st |= h[i].status;
        if (h[i].status && first < 0) first = i;
    }
    if (st & ST_NUMERIC) return fail(TSIM_ERR_NUMERIC, "non-finite state or J <= 0 (instance " + std::to_string(first) + ")");
    if (st & ST_DOMAIN) return fail(TSIM_ERR_DOMAIN, "a particle left the node box (instance " + std::to_string(first) + ")");
    if (st & ST_CAPACITY) return fail(TSIM_ERR_CAPACITY, "a cell block overflowed (instance " + std::to_string(first) + ")");
    if (st & ST_TIMEOUT) return fail(TSIM_ERR_TIMEOUT, "a device wait gave up (instance " + std::to_string(first) + ")");
    return TSIM_OK;
}

extern "C" int tsim_sync(tsim_ctx *c)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    return latched(c);
}

extern "C" int tsim_stats(tsim_ctx *c, tsim_stats_t *out)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    if (!out) return fail(TSIM_ERR_INVALID_ARG, "out is NULL");
    CU(cudaStreamSynchronize(c->stream));
    std::vector<InstState> h(c->n_inst);
    CU(cudaMemcpy(h.data(), c->d.ist, sizeof(InstState) * c->n_inst, cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof(*out));
    out->n_inst = c->n_inst;
    for (int i = 0; i < c->n_inst; ++i) {
        out->passes += h[i].passes_total;
        out->particle_updates += h[i].passes_total * (int64_t)c->hinst[i].n_particles;
        out->status |= h[i].status;
        if (i == 0) out->substeps = h[i].substeps;
        out->spilled += h[i].spilled;
        if (h[i].sp_max > out->spill_max) out->spill_max = h[i].sp_max;
    }
    return TSIM_OK;
}

static int copy_out(tsim_ctx *c, void *dst, const void *src, size_t bytes, int on_device)
{
    CU(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    return TSIM_OK;
}

extern "C" int tsim_read_particles(tsim_ctx *c, int inst, float *x, float *v, float *C, float *F, int n,
                                   int on_device)
{
    int rc = check_ctx(c, inst);
    if (rc) return rc;
    const Inst &I = c->hinst[inst];
    if (n != I.n_particles) return fail(TSIM_ERR_INVALID_ARG, "n must equal the instance's particle count");
    if (!c->have_particles[inst]) return fail(TSIM_ERR_STATE, "no particles written");
    launch_gather(c->d, inst, (long long)I.nblocks * CAP + I.spc, c->par_next, c->stream);
    CU(cudaGetLastError());
    const size_t o = (size_t)I.id0;
    if (x && (rc = copy_out(c, x, c->d.sx + o * 3, sizeof(float) * 3 * n, on_device))) return rc;
    if (v && (rc = copy_out(c, v, c->d.sv + o * 3, sizeof(float) * 3 * n, on_device))) return rc;
    if (C && (rc = copy_out(c, C, c->d.sC + o * 9, sizeof(float) * 9 * n, on_device))) return rc;
    if (F && (rc = copy_out(c, F, c->d.sF + o * 9, sizeof(float) * 9 * n, on_device))) return rc;
    return latched(c);
}

extern "C" int tsim_read_grid(tsim_ctx *c, int inst, float *out, int on_device)
{
    int rc = check_ctx(c, inst);
    if (rc) return rc;
    if (!out) return fail(TSIM_ERR_INVALID_ARG, "out is NULL");
    if (!c->have_particles[inst]) return fail(TSIM_ERR_STATE, "no particles written");
    rc = pending_prologues(c);
    if (rc) return rc;
    const Inst &I = c->hinst[inst];
    rc = copy_out(c, out, c->d.acc + I.node0, sizeof(float4) * (size_t)I.nx * I.ny * I.nz, on_device);
    if (rc) return rc;
    return latched(c);
}

extern "C" int tsim_read_surface(tsim_ctx *c, int inst, float *height, float *normal, int W, int H, float pitch,
                                 int on_device)
{
    int rc = check_ctx(c, inst);
    if (rc) return rc;
    if (W < 1 || H < 1 || (long long)W * H > RO_MAX || !(pitch > 0.f))
        return fail(TSIM_ERR_INVALID_ARG, "need 1 <= W*H <= 2^20 and pitch > 0");
    if (!c->have_particles[inst]) return fail(TSIM_ERR_STATE, "no particles written");
    const Inst &I = c->hinst[inst];
    const size_t WH = (size_t)W * H;
    float *num = c->ro, *den = c->ro + WH, *h = c->ro + 2 * WH, *nrm = c->ro + 3 * WH;
    launch_surface(c->d, inst, (long long)I.nblocks * CAP + I.spc, c->par_next, num, den, h, nrm, W, H, pitch, I.H,
                   c->stream);
    CU(cudaGetLastError());
    if (height && (rc = copy_out(c, height, h, sizeof(float) * WH, on_device))) return rc;
    if (normal && (rc = copy_out(c, normal, nrm, sizeof(float) * WH * 3, on_device))) return rc;
    return latched(c);
}

extern "C" int tsim_read_displacement(tsim_ctx *c, int inst, const float *x_ref, float *u, int W, int H,
                                      float pitch, int on_device)
{
    int rc = check_ctx(c, inst);
    if (rc) return rc;
    if (!x_ref || !u || W < 1 || H < 1 || (long long)W * H > RO_MAX / 2 || !(pitch > 0.f))
        return fail(TSIM_ERR_INVALID_ARG, "need x_ref, u, 1 <= W*H <= 2^19 and pitch > 0");
    if (!c->have_particles[inst]) return fail(TSIM_ERR_STATE, "no particles written");
    const Inst &I = c->hinst[inst];
    const size_t WH = (size_t)W * H;
    const float *xr = x_ref;
    if (!on_device) {       // reference positions go through the id-ordered staging velocity buffer
        CU(cudaMemcpyAsync(c->d.sv + (size_t)I.id0 * 3, x_ref, sizeof(float) * 3 * (size_t)I.n_particles,
                           cudaMemcpyHostToDevice, c->stream));
        xr = c->d.sv + (size_t)I.id0 * 3;
    }
    float *acc = c->ro, *uf = c->ro + 4 * WH;
    launch_surface_disp(c->d, inst, (long long)I.nblocks * CAP + I.spc, c->par_next, xr, acc, uf, W, H, pitch,
                        c->stream);
    CU(cudaGetLastError());
    rc = copy_out(c, u, uf, sizeof(float) * 3 * WH, on_device);
    if (rc) return rc;
    return latched(c);
}

extern "C" int tsim_read_indenter_height(tsim_ctx *c, int inst, float *h, int W, int H, float pitch, float clip,
                                         int on_device)
{
    int rc = check_ctx(c, inst);
    if (rc) return rc;
    if (!h || W < 1 || H < 1 || (long long)W * H > RO_MAX || !(pitch > 0.f) || !(clip > 0.f))
        return fail(TSIM_ERR_INVALID_ARG, "need h, 1 <= W*H <= 2^20, pitch > 0, clip > 0");
    launch_indenter_height(c->d, inst, c->ro, W, H, pitch, clip, c->stream);
    CU(cudaGetLastError());
    rc = copy_out(c, h, c->ro, sizeof(float) * (size_t)W * H, on_device);
    if (rc) return rc;
    return latched(c);
}

extern "C" int tsim_read_markers(tsim_ctx *c, int inst, const int32_t *ids, int m, float *xyz, int on_device)
{
    int rc = check_ctx(c, inst);
    if (rc) return rc;
    if (!ids || !xyz || m < 1 || m > MARK_MAX) return fail(TSIM_ERR_INVALID_ARG, "need 1..4096 ids");
    if (!c->have_particles[inst]) return fail(TSIM_ERR_STATE, "no particles written");
    const Inst &I = c->hinst[inst];
    CU(cudaMemcpyAsync(c->ids, ids, sizeof(int) * m, cudaMemcpyHostToDevice, c->stream));
    launch_gather(c->d, inst, (long long)I.nblocks * CAP + I.spc, c->par_next, c->stream);
    launch_pick(c->d, inst, c->ids, m, c->pick, c->stream);
    CU(cudaGetLastError());
    rc = copy_out(c, xyz, c->pick, sizeof(float) * 3 * m, on_device);
    if (rc) return rc;
    return latched(c);
}

extern "C" int tsim_read_log(tsim_ctx *c, int inst, int32_t *passes, int32_t *calib, int n)
{
    int rc = check_ctx(c, inst);
    if (rc) return rc;
    if (n < 0 || n > LOGN) return fail(TSIM_ERR_INVALID_ARG, "n must be 0..32768");
    CU(cudaStreamSynchronize(c->stream));
    std::vector<int2> lg(LOGN);
    InstState st;
    CU(cudaMemcpy(lg.data(), c->d.log + (size_t)inst * LOGN, sizeof(int2) * LOGN, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(&st, c->d.ist + inst, sizeof(InstState), cudaMemcpyDeviceToHost));
    const long long total = st.substeps;
    for (int a = 0; a < n; ++a) {
        long long s = total - n + a;
        int2 e = s >= 0 ? lg[s % LOGN] : make_int2(0, -1);
        if (passes) passes[a] = e.x;
        if (calib) calib[a] = e.y;
    }
    return TSIM_OK;
}

extern "C" int tsim_use_graph(tsim_ctx *c, int enable)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    CU(cudaStreamSynchronize(c->stream));
    c->use_graph = enable != 0;
    return TSIM_OK;
}

extern "C" int tsim_profile(tsim_ctx *c, int enable)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    CU(cudaStreamSynchronize(c->stream));
    for (auto &g : c->chunks)
        if ((rc = harvest(c, g))) return rc;
    if ((rc = harvest_stream(c))) return rc;
    if ((enable != 0) != c->profile) invalidate_graphs(c);
    c->profile = enable != 0;
    return TSIM_OK;
}

extern "C" int tsim_pass_time(tsim_ctx *c, int64_t *launches, double *commit_ms, double *loop_ms)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    CU(cudaStreamSynchronize(c->stream));
    for (auto &g : c->chunks)
        if ((rc = harvest(c, g))) return rc;
    if ((rc = harvest_stream(c))) return rc;
    if (launches) *launches = c->prof_launches;
    if (commit_ms) *commit_ms = c->prof_ms;
    if (loop_ms) *loop_ms = c->prof_loop_ms;
    c->prof_launches = 0;
    c->prof_ms = 0.0;
    c->prof_loop_ms = 0.0;
    return TSIM_OK;
}

extern "C" int tsim_kernel_time(tsim_ctx *c, int64_t *launches, double *total_ms)
{
    return tsim_pass_time(c, launches, total_ms, nullptr);
}

// ---------------------------------------------------------------- execution configuration

static bool valid_tuning(const tsim_tuning_t *t)
{
    return t && (t->grid_threads == 128 || t->grid_threads == 256 || t->grid_threads == 512) &&
           (t->grid_flat == 0 || t->grid_flat == 1) && t->graph_chunk >= 1 && t->graph_chunk <= 200;
}

static void apply_tuning(tsim_ctx *c, int threads, int flat, int chunk)
{
    if (threads != c->grid_threads || flat != c->grid_flat || chunk != c->chunk_len) invalidate_graphs(c);
    c->grid_threads = threads;
    c->grid_flat = flat;
    c->chunk_len = chunk;
}

extern "C" int tsim_set_tuning(tsim_ctx *c, const tsim_tuning_t *t)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    if (!valid_tuning(t))
        return fail(TSIM_ERR_INVALID_ARG, "tuning: grid_threads in {128, 256, 512}, grid_flat in {0, 1}, "
                                          "1 <= graph_chunk <= 200");
    CU(cudaStreamSynchronize(c->stream));
    for (auto &g : c->chunks)
        if ((rc = harvest(c, g))) return rc;
    apply_tuning(c, t->grid_threads, t->grid_flat, t->graph_chunk);
    return TSIM_OK;
}

extern "C" int tsim_get_tuning(tsim_ctx *c, tsim_tuning_t *out)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    if (!out) return fail(TSIM_ERR_INVALID_ARG, "out is NULL");
    out->grid_threads = c->grid_threads;
    out->grid_flat = c->grid_flat;
    out->graph_chunk = c->chunk_len;
    out->us_per_mupdate = c->tuned_us;
    return TSIM_OK;
}

// particle-updates done so far (sum over instances of passes x particles); synchronises
static int updates_so_far(tsim_ctx *c, double *out)
{
    CU(cudaStreamSynchronize(c->stream));
    std::vector<InstState> h(c->n_inst);
    CU(cudaMemcpy(h.data(), c->d.ist, sizeof(InstState) * c->n_inst, cudaMemcpyDeviceToHost));
    double u = 0.0;
    for (int i = 0; i < c->n_inst; ++i) u += (double)h[i].passes_total * c->hinst[i].n_particles;
    *out = u;
    return TSIM_OK;
}

// n substeps with the given configuration, timed with events on the stream
// (graph executables are built before the first event)
static int timed_window(tsim_ctx *c, int threads, int flat, int chunk, int n, double *ms, double *upd)
{
    for (auto &g : c->chunks) {
        int rc = harvest(c, g);
        if (rc) return rc;
    }
    apply_tuning(c, threads, flat, chunk);
    if (c->use_graph) {
        int rc = ensure_chunks(c);
        if (rc) return rc;
    }
    double u0 = 0.0, u1 = 0.0;
    int rc = updates_so_far(c, &u0);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    cudaEventRecord(e0, c->stream);
    rc = step_n(c, n);
    cudaEventRecord(e1, c->stream);
    if (rc == TSIM_OK) rc = updates_so_far(c, &u1);
    float t = 0.f;
    if (rc == TSIM_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
        rc = fail(TSIM_ERR_CUDA, "autotune: event timing failed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *ms += t;
    *upd += u1 - u0;
    return latched(c);
}

// Online autotuning: the n substeps are the simulation's own (the state
// advances as with tsim_step(n); the candidates differ only in how the same
// kernels are launched).  Two interleaved rounds time the six grid-update
// launch shapes on windows of equal length, then the three graph chunk
// lengths (graph mode) with the best shape; the fastest per particle-update
// is kept and the rest of the n substeps run with it.
extern "C" int tsim_autotune(tsim_ctx *c, int n, tsim_tuning_t *out)
{
    int rc = check_ctx(c, 0);
    if (rc) return rc;
    static const int shapes[6][2] = {{128, 0}, {256, 0}, {512, 0}, {128, 1}, {256, 1}, {512, 1}};
    static const int chunks[3] = {10, 20, 40};
    const int rounds = 2, nwin = 6 * rounds + (c->use_graph ? 3 : 0);
    int win = n / nwin;
    if (c->use_graph) win = win / 40 * 40;           // whole graph launches for every chunk length
    if (win < (c->use_graph ? 40 : 2))
        return fail(TSIM_ERR_INVALID_ARG, std::string("autotune needs n >= ") +
                                              std::to_string(nwin * (c->use_graph ? 40 : 2)) + " substeps");
    rc = check_steppable(c);
    if (rc) return rc;
    const int chunk0 = c->chunk_len;
    double ms[6] = {0}, upd[6] = {0};
    for (int r = 0; r < rounds; ++r)
        for (int k = 0; k < 6; ++k) {
            const int kk = (r & 1) ? 5 - k : k;      // alternate the order between rounds
            rc = timed_window(c, shapes[kk][0], shapes[kk][1], chunk0, win, &ms[kk], &upd[kk]);
            if (rc) return rc;
        }
    int best = 0;
    for (int k = 1; k < 6; ++k)
        if (ms[k] * upd[best] < ms[best] * upd[k]) best = k;
    double best_us = 1e3 * ms[best] / std::max(upd[best] * 1e-6, 1e-30);
    int best_chunk = chunk0;
    if (c->use_graph) {
        double cms[3] = {0}, cupd[3] = {0};
        int bc = 0;
        for (int k = 0; k < 3; ++k) {
            rc = timed_window(c, shapes[best][0], shapes[best][1], chunks[k], win, &cms[k], &cupd[k]);
            if (rc) return rc;
            if (k > 0 && cms[k] * cupd[bc] < cms[bc] * cupd[k]) bc = k;
        }
        best_chunk = chunks[bc];
        best_us = 1e3 * cms[bc] / std::max(cupd[bc] * 1e-6, 1e-30);
    }
    apply_tuning(c, shapes[best][0], shapes[best][1], best_chunk);
    c->tuned_us = (float)best_us;
    const int rest = n - nwin * win;
    if (rest > 0) {
        rc = step_n(c, rest);
        if (rc) return rc;
    }
    if (out) tsim_get_tuning(c, out);
    return latched(c);
}
