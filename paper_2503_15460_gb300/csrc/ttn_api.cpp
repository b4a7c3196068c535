// libttn C ABI (declarations and documentation in include/ttn.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <set>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ttn.h"
#include "ttn_ctx.hpp"
#include "ttn_launch.h"
#include "ttn_plan.hpp"

using ttn::cplx;

using ttn::DevProgram;

namespace {

thread_local std::string g_create_error;

ttn_status fail(ttn_ctx* c, ttn_status s, const std::string& msg) {
    if (c) {
        c->err = msg;
        if (s == TTN_E_CUDA || s == TTN_E_NOCONV || s == TTN_E_TIMEOUT) c->failed = true;
    } else {
        g_create_error = msg;
    }
    return s;
}

ttn_status cuda_fail(ttn_ctx* c, cudaError_t e, const char* what) {
    return fail(c, TTN_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

// Convert host complex128 data into the bulk element type.
std::vector<char> to_bulk(const cplx* src, size_t n, size_t esz) {
    std::vector<char> out(n * esz);
    if (esz == 16) {
        std::memcpy(out.data(), src, n * 16);
    } else {
        float* f = (float*)out.data();
        for (size_t i = 0; i < n; ++i) { f[2 * i] = (float)src[i].real(); f[2 * i + 1] = (float)src[i].imag(); }
    }
    return out;
}

void from_bulk(const char* src, size_t n, size_t esz, cplx* dst) {
    if (esz == 16) { std::memcpy(dst, src, n * 16); return; }
    const float* f = (const float*)src;
    for (size_t i = 0; i < n; ++i) dst[i] = cplx(f[2 * i], f[2 * i + 1]);
}

}  // namespace

TtnInstance ttn::make_instance(ttn_ctx* c, const DevProgram& p) {
    TtnInstance in{};
    in.ops = p.d_ops;
    in.n_ops = p.n_ops;
    in.n_slots = (int)c->plan.slots.size();
    in.entries = c->d_entries;
    in.slots = c->d_slots;
    in.work = c->d_state + c->plan.work_off;
    in.smax = c->plan.smax;
    in.status = (int*)(c->d_state + c->plan.status_off);
    in.steps_done = (int*)(c->d_state + c->plan.steps_off);
    in.stamps = (unsigned long long*)(c->d_state + c->plan.stamps_off);
    in.flops = (double*)(c->d_state + c->plan.flops_off);
    in.op_cycles = (unsigned long long*)(c->d_state + c->plan.cycles_off);
    in.ktol = c->ktol > 0 ? c->ktol : (c->precision == TTN_MIXED ? 1e-10 : 1e-13);
    in.qtol = c->qtol > 0 ? c->qtol : 1e-10;
    in.kmax = c->kmax;
    in.spawn_out = (double*)(c->d_state + c->plan.spawn_out_off);
    in.spawn_ws = c->d_state + c->plan.spawn_ws_off;
    in.spawn_kmax = c->plan.spawn_kmax;
    in.use_tc = 0;
    for (int n = 0; n <= TTN_MAXCHI; ++n) {
        in.mp_variant[n] = c->mp_variant[n];
        in.use_tc |= c->mp_variant[n] == 2 && c->precision == TTN_MIXED;
    }
    return in;
}

ttn_status ttn::ctx_fail(ttn_ctx* c, ttn_status s, const std::string& msg) { return fail(c, s, msg); }

bool ttn::ctx_uses_tc(const ttn_ctx* c) {
    if (c->precision != TTN_MIXED) return false;
    for (int n = 0; n <= TTN_MAXCHI; ++n)
        if (c->mp_variant[n] == 2) return true;
    return false;
}

int ttn::ctx_cluster(const ttn_ctx* c) {
    const int need = c->plan.max_chi > kSoloMaxDim ? 2 : 1;
    if (c->cluster_req > 0) return std::max(c->cluster_req, need);
    int64_t per = c->plan.smax / 4096;
    int k = 1;
    while (k * 2 <= per && k < TTN_MAX_CLUSTER) k *= 2;
    return std::max(k, need);
}

namespace {

using ttn::make_instance;

cudaError_t dev_alloc(ttn_ctx* c, char** p, size_t n) {
    return c->pooled ? cudaMallocAsync((void**)p, n, c->stream) : cudaMalloc((void**)p, n);
}

void dev_free(ttn_ctx* c, char* p) {
    if (!p) return;
    if (c->pooled) cudaFreeAsync(p, c->stream);
    else cudaFree(p);
}

// Allocation failure: TTN_E_OOM, context left as it was; other errors fail it.
ttn_status alloc_fail(ttn_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(c, TTN_E_OOM, std::string(what) + ": out of device memory");
    }
    return cuda_fail(c, e, what);
}

// Layout of the operator arena: slot storage, slot table, entries, ops, instance.
struct OpsLayout {
    size_t slot_bytes, off_table, off_entries, off_ops, off_inst, total;
};

OpsLayout ops_layout(const ttn::Plan& P) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    OpsLayout L{};
    for (auto& s : P.slots) L.slot_bytes = std::max(L.slot_bytes, (size_t)s.off + (size_t)s.rows * s.cols * P.esz);
    L.slot_bytes = al(L.slot_bytes);
    size_t n_ops_total = P.init_prog.ops.size() + P.step_prog.ops.size() + P.norm_energy_prog.ops.size() +
                         P.spawn_prog.ops.size() + P.ground_prog.ops.size() + P.setpop_prog.ops.size();
    for (auto& p : P.rdm_prog) n_ops_total += p.ops.size();
    for (auto& p : P.vac_prog) n_ops_total += p.ops.size();
    for (auto& p : P.to_root_prog) n_ops_total += p.ops.size();
    L.off_table = L.slot_bytes;
    L.off_entries = al(L.off_table + P.slots.size() * sizeof(TtnSlot));
    L.off_ops = al(L.off_entries + std::max<size_t>(1, P.entries.size()) * sizeof(TtnEntry));
    L.off_inst = al(L.off_ops + std::max<size_t>(1, n_ops_total) * sizeof(TtnOp));
    L.total = al(L.off_inst + sizeof(TtnInstance));
    return L;
}

ttn_status check_status(ttn_ctx* c) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, c->d_state + c->plan.status_off, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status copy");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    if (st == 4) return fail(c, TTN_E_NOCONV, "Krylov exponential did not converge");
    if (st == 5) return fail(c, TTN_E_TIMEOUT, "device wait timed out");
    if (st != 0) return fail(c, TTN_E_CUDA, "device reported status " + std::to_string(st));
    return TTN_OK;
}

ttn_status run_program(ttn_ctx* c, const DevProgram& p, double dt, int nrep) {
    if (p.n_ops == 0 || nrep == 0) return TTN_OK;
    TtnInstance in = make_instance(c, p);
    CK(cudaMemcpyAsync(c->d_inst, &in, sizeof(in), cudaMemcpyHostToDevice, c->stream), "instance upload");
    int e = ttn_launch_program(c->precision, ttn::ctx_cluster(c), c->d_inst, 1, dt, nrep, c->stream,
                               ttn::ctx_uses_tc(c));
    if (e != 0) return cuda_fail(c, (cudaError_t)e, "kernel launch");
    return check_status(c);
}

ttn_status check_status_spawn(ttn_ctx* c, bool* hit) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, c->d_state + c->plan.status_off, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status copy");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    *hit = st == TTN_STATUS_SPAWN_HIT;
    if (*hit) return TTN_OK;
    if (st == 4) return fail(c, TTN_E_NOCONV, "Krylov exponential did not converge");
    if (st == TTN_STATUS_SPAWN_SPACE)
        return fail(c, TTN_E_INVALID, "subspace expansion: a bond has more than " +
                    std::to_string(TTN_SPAWN_MAX_CHANNELS) + " up channels or a channel space above " +
                    std::to_string(TTN_SPAWN_MAX_K));
    if (st != 0) return fail(c, TTN_E_CUDA, "device reported status " + std::to_string(st));
    return TTN_OK;
}

void free_ops(ttn_ctx* c) {
    dev_free(c, c->d_ops);
    c->d_ops = nullptr;
    c->ops_bytes = 0;
    c->d_slots = nullptr;
    c->d_entries = nullptr;
    c->init_p = c->step_p = c->ne_p = c->spawn_p = c->ground_p = c->setpop_p = DevProgram();
    c->rdm_p.clear(); c->vac_p.clear(); c->to_root_p.clear();
    c->d_inst = nullptr;
}

// Allocate and fill the operator arena for the current plan.
ttn_status upload_ops(ttn_ctx* c) {
    ttn::Plan& P = c->plan;
    const OpsLayout L = ops_layout(P);
    const size_t off_table = L.off_table, off_entries = L.off_entries, off_ops = L.off_ops, off_inst = L.off_inst;
    const size_t total = L.total;
    if (!(c->d_ops && c->ops_bytes == total)) {
        // a layout of the same size (new coefficients, same structure) reuses the arena
        free_ops(c);
        char* arena = nullptr;
        cudaError_t ae = dev_alloc(c, &arena, total);
        if (ae != cudaSuccess) return alloc_fail(c, ae, "device allocation (operators)");
        c->d_ops = arena;
        c->ops_bytes = total;
    }
    c->rdm_p.clear(); c->vac_p.clear(); c->to_root_p.clear();
    std::vector<char> host(total, 0);
    // constant slots
    for (auto& s : P.slots)
        if (s.constant) {
            auto b = to_bulk(s.data.data(), s.data.size(), P.esz);
            std::memcpy(host.data() + s.off, b.data(), b.size());
        }
    // slot table
    std::vector<TtnSlot> table(P.slots.size());
    for (size_t i = 0; i < P.slots.size(); ++i) {
        table[i].ptr = c->d_ops + P.slots[i].off;
        table[i].rows = P.slots[i].rows;
        table[i].cols = P.slots[i].cols;
    }
    std::memcpy(host.data() + off_table, table.data(), table.size() * sizeof(TtnSlot));
    std::memcpy(host.data() + off_entries, P.entries.data(), P.entries.size() * sizeof(TtnEntry));
    // programs
    size_t cur = off_ops;
    auto link = [&](const ttn::Program& p) {
        DevProgram d;
        d.d_ops = (TtnOp*)(c->d_ops + cur);
        d.n_ops = (int)p.ops.size();
        for (auto& s : p.ops) {
            TtnOp o = s.op;
            o.a = s.a_off >= 0 ? (void*)(c->d_state + s.a_off) : nullptr;
            o.b = s.b_off >= 0 ? (void*)(c->d_state + s.b_off) : nullptr;
            o.out = s.out_off >= 0 ? (double*)(c->d_state + s.out_off) : nullptr;
            if (o.type == TTN_OP_SPAWN) o.c = o.b;      // the child tensor
            else o.c = s.c_off >= 0 ? (void*)(c->d_state + s.c_off) : nullptr;   // ENV: ket tensor
            std::memcpy(host.data() + cur, &o, sizeof(TtnOp));
            cur += sizeof(TtnOp);
        }
        return d;
    };
    c->init_p = link(P.init_prog);
    c->step_p = link(P.step_prog);
    c->ne_p = link(P.norm_energy_prog);
    c->spawn_p = link(P.spawn_prog);
    c->ground_p = link(P.ground_prog);
    c->setpop_p = link(P.setpop_prog);
    for (auto& p : P.rdm_prog) c->rdm_p.push_back(link(p));
    for (auto& p : P.vac_prog) c->vac_p.push_back(link(p));
    for (auto& p : P.to_root_prog) c->to_root_p.push_back(link(p));
    c->d_slots = (TtnSlot*)(c->d_ops + off_table);
    c->d_entries = (TtnEntry*)(c->d_ops + off_entries);
    c->d_inst = (TtnInstance*)(c->d_ops + off_inst);
    CK(cudaMemcpyAsync(c->d_ops, host.data(), total, cudaMemcpyHostToDevice, c->stream), "operator upload");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    return TTN_OK;
}

ttn_status upload_state(ttn_ctx* c, const std::vector<std::vector<cplx>>& A);

// Node tensors of a resident context, copied to the host.
ttn_status download_state(ttn_ctx* c, std::vector<std::vector<cplx>>& A) {
    std::vector<char> raw(c->plan.bond_off);
    CK(cudaMemcpyAsync(raw.data(), c->d_state, raw.size(), cudaMemcpyDeviceToHost, c->stream), "state copy");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    A.assign(c->tree.n, {});
    for (int u = 0; u < c->tree.n; ++u) {
        const cplx* src = (const cplx*)(raw.data() + c->plan.tensor_off[u]);
        A[u].assign(src, src + c->plan.nset * c->tree.size[u]);     // all set blocks
    }
    return TTN_OK;
}

// Grow the bond of `child` by the p functions in U (NJ x p, column j of the
// new block = U[j*NJ ..]): append them to the child's tensor, zero-pad the
// parent's index, and rebuild plan, arenas, centre position and
// environments for the new bond dimensions (paper Sec. II.D: the state is
// unchanged by the padding).
ttn_status grow_bond(ttn_ctx* c, int child, int p, const std::vector<cplx>& U) {
    ttn::Tree& t = c->tree;
    const int z = t.parent[child];
    const int k = (int)(std::find(t.ch[z].begin(), t.ch[z].end(), child) - t.ch[z].begin());
    std::vector<std::vector<cplx>> A;
    ttn_status ds = download_state(c, A);
    if (ds) return ds;
    const int chi = t.bond[child];
    const int64_t NJ = t.size[child] / chi;
    // child: [NJ x chi] -> [NJ x (chi + p)]
    std::vector<cplx> Ac(NJ * (chi + p));
    for (int64_t J = 0; J < NJ; ++J) {
        for (int n = 0; n < chi; ++n) Ac[J * (chi + p) + n] = A[child][J * chi + n];
        for (int j = 0; j < p; ++j) Ac[J * (chi + p) + chi + j] = U[(size_t)j * NJ + J];
    }
    // parent: index k grows from chi to chi + p with zeros
    const auto& dz = t.dims[z];
    int64_t Lk = 1, Rk = 1;
    for (int j = 0; j < k; ++j) Lk *= dz[j];
    for (size_t j = k + 1; j < dz.size(); ++j) Rk *= dz[j];
    std::vector<cplx> Az(Lk * (chi + p) * Rk, 0.0);
    for (int64_t l = 0; l < Lk; ++l)
        for (int n = 0; n < chi; ++n)
            for (int64_t r = 0; r < Rk; ++r) Az[(l * (chi + p) + n) * Rk + r] = A[z][(l * chi + n) * Rk + r];
    A[child].swap(Ac);
    A[z].swap(Az);
    std::vector<int> bond = t.bond;
    bond[child] = chi + p;
    ttn::Tree nt;
    std::string msg = ttn::build_tree(t.n, t.parent.data(), t.phys.data(), bond.data(), nt);
    if (!msg.empty()) return fail(c, TTN_E_STATE, "bond growth produced an invalid tree: " + msg);
    ttn::Plan P;
    msg = ttn::make_plan(nt, &c->ham, c->precision, P);
    if (!msg.empty()) return fail(c, TTN_E_STATE, msg);
    char* fresh = nullptr;
    cudaError_t ae = dev_alloc(c, &fresh, P.total_bytes);
    if (ae != cudaSuccess) { c->failed = true; return alloc_fail(c, ae, "device allocation (state)"); }
    dev_free(c, c->d_state);
    c->d_state = fresh;
    c->state_bytes = P.total_bytes;
    CK(cudaMemsetAsync(c->d_state, 0, c->state_bytes, c->stream), "memset");
    c->tree = nt;
    c->plan = P;
    ttn_status s = upload_ops(c);
    if (s) { c->failed = true; return s; }
    s = upload_state(c, A);
    if (s) return s;
    if (z > 0) { s = run_program(c, c->to_root_p[z], 0.0, 1); if (s) return s; }
    return run_program(c, c->init_p, 0.0, 1);
}

// One expansion pass: run the spawn program until it finishes without a hit.
ttn_status expand_pass(ttn_ctx* c, double dt, double eps, int chi_max) {
    if (c->plan.nset > 1)
        return fail(c, TTN_E_INVALID, "subspace expansion is for single-set states (the paper leaves the multi-set case open)");
    for (int guard = 0; guard < 100000; ++guard) {
        if (c->spawn_p.n_ops == 0) return TTN_OK;
        TtnInstance in = make_instance(c, c->spawn_p);
        in.chi_max = chi_max; in.spawn_eps = eps; in.spawn_dt = dt;
        CK(cudaMemcpyAsync(c->d_inst, &in, sizeof(in), cudaMemcpyHostToDevice, c->stream), "instance upload");
        int e = ttn_launch_program(c->precision, ttn::ctx_cluster(c), c->d_inst, 1, dt, 1, c->stream,
                                   ttn::ctx_uses_tc(c));
        if (e != 0) return cuda_fail(c, (cudaError_t)e, "kernel launch");
        bool hit = false;
        ttn_status s = check_status_spawn(c, &hit);
        if (s) return s;
        if (!hit) return TTN_OK;
        double hdr[4];
        CK(cudaMemcpyAsync(hdr, c->d_state + c->plan.spawn_out_off, sizeof(hdr), cudaMemcpyDeviceToHost, c->stream), "spawn copy");
        CK(cudaStreamSynchronize(c->stream), "stream synchronize");
        const int child = (int)hdr[1], p = (int)hdr[2];
        const int64_t NJ = (int64_t)hdr[3];
        std::vector<cplx> U((size_t)NJ * p);
        CK(cudaMemcpyAsync(U.data(), c->d_state + c->plan.spawn_out_off + 8 * (4 + TTN_SPAWN_MAX_NEW), U.size() * 16,
                           cudaMemcpyDeviceToHost, c->stream), "spawn copy");
        int zero = 0;
        CK(cudaMemcpyAsync(c->d_state + c->plan.status_off, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream), "status reset");
        CK(cudaStreamSynchronize(c->stream), "stream synchronize");
        s = grow_bond(c, child, p, U);
        if (s) return s;
        c->spawned += p;
    }
    return fail(c, TTN_E_STATE, "expansion pass did not terminate");
}

ttn_status upload_state(ttn_ctx* c, const std::vector<std::vector<cplx>>& A) {
    std::vector<char> host(c->plan.bond_off, 0);
    for (int z = 0; z < c->tree.n; ++z) {
        std::memcpy(host.data() + c->plan.tensor_off[z], A[z].data(), A[z].size() * 16);
    }
    CK(cudaMemcpyAsync(c->d_state, host.data(), host.size(), cudaMemcpyHostToDevice, c->stream), "state upload");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    return TTN_OK;
}

ttn_status usable(ttn_ctx* c) {
    if (!c) return TTN_E_INVALID;
    if (c->failed) return fail(c, TTN_E_STATE, "context is in a failed state: " + c->err);
    if (!c->resident) return TTN_OK;      // host-resident: no device work until materialised
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return TTN_OK;
}

// usable() and resident on the device.
ttn_status ready(ttn_ctx* c) {
    ttn_status u = usable(c);
    if (u) return u;
    if (!c->resident) {
        cudaError_t e = cudaSetDevice(c->device);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    }
    return ttn::ctx_materialize(c);
}

// Tensors given by the caller: to the device (resident) or kept on the host.
ttn_status take_state(ttn_ctx* c, std::vector<std::vector<cplx>>& A) {
    if (!c->resident) {
        c->host_A.swap(A);
        return TTN_OK;
    }
    ttn_status s = upload_state(c, A);
    if (s) return s;
    if (c->has_h) return run_program(c, c->init_p, 0.0, 1);
    return TTN_OK;
}

ttn_status create_ctx(int n_nodes, const int* parent, const int* phys_dim, const int* bond_dim, int precision,
                      bool on_host, ttn_ctx** out) {
    if (!out) return fail(nullptr, TTN_E_INVALID, "out is NULL");
    *out = nullptr;
    if (precision != TTN_FP64 && precision != TTN_MIXED) return fail(nullptr, TTN_E_INVALID, "precision must be TTN_FP64 or TTN_MIXED");
    ttn::Tree t;
    std::string msg = ttn::build_tree(n_nodes, parent, phys_dim, bond_dim, t);
    if (!msg.empty()) return fail(nullptr, TTN_E_INVALID, msg);
    ttn_ctx* c = new (std::nothrow) ttn_ctx();
    if (!c) return fail(nullptr, TTN_E_OOM, "host allocation failed");
    c->precision = precision;
    c->tree = t;
    cudaGetDevice(&c->device);
    ttn::make_plan(c->tree, nullptr, precision, c->plan);
    std::vector<std::vector<cplx>> vecs(t.n), A;
    for (int z = 0; z < t.n; ++z)
        if (t.leaf(z)) { vecs[z].assign(t.phys[z], 0.0); vecs[z][0] = 1.0; }
    ttn::product_state(t, vecs, A);
    if (on_host) {
        c->resident = false;
        c->pooled = true;
        c->host_A.swap(A);
        *out = c;
        return TTN_OK;
    }
    cudaError_t e = cudaMalloc(&c->d_state, c->plan.total_bytes);
    if (e != cudaSuccess) {
        g_create_error = std::string("cudaMalloc (state): ") + cudaGetErrorString(e);
        delete c;
        return e == cudaErrorMemoryAllocation ? TTN_E_OOM : TTN_E_CUDA;
    }
    c->state_bytes = c->plan.total_bytes;
    cudaMemset(c->d_state, 0, c->state_bytes);
    ttn_status s = upload_ops(c);
    if (s != TTN_OK) { g_create_error = c->err; ttn_destroy(c); return s; }
    s = upload_state(c, A);
    if (s != TTN_OK) { g_create_error = c->err; ttn_destroy(c); return s; }
    *out = c;
    return TTN_OK;
}

}  // namespace

size_t ttn::ctx_footprint(const ttn_ctx* c) { return (size_t)c->plan.total_bytes + ops_layout(c->plan).total; }

ttn_status ttn::ctx_materialize(ttn_ctx* c) {
    if (c->resident) return TTN_OK;
    char* st = nullptr;
    cudaError_t ae = dev_alloc(c, &st, c->plan.total_bytes);
    if (ae != cudaSuccess) return alloc_fail(c, ae, "device allocation (state)");
    c->d_state = st;
    c->state_bytes = c->plan.total_bytes;
    c->resident = true;
    CK(cudaMemsetAsync(c->d_state, 0, c->state_bytes, c->stream), "memset");
    ttn_status s = upload_ops(c);
    if (s) {
        // give the memory back and stay on the host
        free_ops(c);
        dev_free(c, c->d_state);
        c->d_state = nullptr; c->state_bytes = 0; c->resident = false;
        return s;
    }
    const int steps = (int)c->saved_steps;
    const double flops[2] = {c->saved_flops, c->saved_flops64};
    CK(cudaMemcpyAsync(c->d_state + c->plan.steps_off, &steps, sizeof(int), cudaMemcpyHostToDevice, c->stream), "counter upload");
    CK(cudaMemcpyAsync(c->d_state + c->plan.flops_off, flops, sizeof(flops), cudaMemcpyHostToDevice, c->stream), "counter upload");
    s = upload_state(c, c->host_A);     // synchronises the stream
    if (s) return s;
    c->host_A.clear();
    c->host_A.shrink_to_fit();
    if (c->has_h) return run_program(c, c->init_p, 0.0, 1);
    return TTN_OK;
}

ttn_status ttn::ctx_evict(ttn_ctx* c) {
    if (!c->resident) return TTN_OK;
    std::vector<std::vector<cplx>> A;
    ttn_status s = download_state(c, A);
    if (s) return s;
    int steps = 0;
    double flops[2] = {0.0, 0.0};
    CK(cudaMemcpyAsync(&steps, c->d_state + c->plan.steps_off, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "counter copy");
    CK(cudaMemcpyAsync(flops, c->d_state + c->plan.flops_off, sizeof(flops), cudaMemcpyDeviceToHost, c->stream), "counter copy");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    free_ops(c);
    dev_free(c, c->d_state);
    c->d_state = nullptr;
    c->state_bytes = 0;
    if (c->d_batch) cudaFree(c->d_batch);
    c->d_batch = nullptr;
    c->batch_cap = 0;
    c->host_A.swap(A);
    c->saved_steps = steps;
    c->saved_flops = flops[0];
    c->saved_flops64 = flops[1];
    c->resident = false;
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    return TTN_OK;
}

namespace {

// Checkpoint byte stream: little helpers over a growing buffer / a cursor.
struct Writer {
    std::vector<char> b;
    template <class T> void put(const T& v) { const char* p = (const char*)&v; b.insert(b.end(), p, p + sizeof(T)); }
    template <class T> void put_vec(const std::vector<T>& v) {
        put<int64_t>((int64_t)v.size());
        const char* p = (const char*)v.data();
        b.insert(b.end(), p, p + v.size() * sizeof(T));
    }
};
struct Reader {
    const char* p;
    size_t left;
    bool ok = true;
    template <class T> T get() {
        T v{};
        if (left < sizeof(T)) { ok = false; return v; }
        std::memcpy(&v, p, sizeof(T)); p += sizeof(T); left -= sizeof(T);
        return v;
    }
    template <class T> std::vector<T> get_vec(int64_t max_n) {
        const int64_t n = get<int64_t>();
        std::vector<T> v;
        if (!ok || n < 0 || n > max_n || (size_t)n * sizeof(T) > left) { ok = false; return v; }
        v.resize((size_t)n);
        std::memcpy(v.data(), p, (size_t)n * sizeof(T)); p += n * sizeof(T); left -= n * sizeof(T);
        return v;
    }
};
const uint32_t kCkptMagic = 0x314E5454u;   // "TTN1"
// A multi-set checkpoint: after the Hamiltonian, the set count and every
// term's set pair; each node's tensor holds all set blocks (set 0 first).
const uint32_t kCkptMagicSets = 0x324E5454u;   // "TTN2"

}  // namespace

extern "C" {

ttn_status ttn_create(int n_nodes, const int* parent, const int* phys_dim, const int* bond_dim, int precision,
                      ttn_ctx** out) {
    return create_ctx(n_nodes, parent, phys_dim, bond_dim, precision, false, out);
}

ttn_status ttn_create_host(int n_nodes, const int* parent, const int* phys_dim, const int* bond_dim, int precision,
                           ttn_ctx** out) {
    return create_ctx(n_nodes, parent, phys_dim, bond_dim, precision, true, out);
}

ttn_status ttn_materialize(ttn_ctx* c) { return ready(c); }

ttn_status ttn_evict(ttn_ctx* c) {
    ttn_status u = usable(c); if (u) return u;
    return ttn::ctx_evict(c);
}

ttn_status ttn_footprint(const ttn_ctx* c, size_t* bytes) {
    if (!c || !bytes) return TTN_E_INVALID;
    *bytes = ttn::ctx_footprint(c);
    return TTN_OK;
}

ttn_status ttn_set_state(ttn_ctx* c, const ttn_c128* tensors, const int64_t* offsets) {
    ttn_status u = usable(c); if (u) return u;
    if (c->plan.nset > 1) return fail(c, TTN_E_INVALID, "the state is multi-set: use ttn_set_multiset_state");
    if (!tensors || !offsets) return fail(c, TTN_E_INVALID, "null tensors / offsets");
    std::vector<std::vector<cplx>> A(c->tree.n);
    for (int z = 0; z < c->tree.n; ++z) {
        if (offsets[z + 1] - offsets[z] != c->tree.size[z])
            return fail(c, TTN_E_INVALID, "tensor " + std::to_string(z) + " has the wrong size");
        const cplx* p = (const cplx*)(tensors + offsets[z]);
        A[z].assign(p, p + c->tree.size[z]);
        for (auto& v : A[z])
            if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) return fail(c, TTN_E_INVALID, "non-finite tensor entry");
    }
    return take_state(c, A);
}

ttn_status ttn_set_product_state(ttn_ctx* c, const ttn_c128* leaf_vecs, const int64_t* leaf_offsets) {
    ttn_status u = usable(c); if (u) return u;
    if (c->plan.nset > 1) return fail(c, TTN_E_INVALID, "the state is multi-set: use ttn_set_multiset_state");
    if (!leaf_vecs || !leaf_offsets) return fail(c, TTN_E_INVALID, "null leaf vectors");
    std::vector<std::vector<cplx>> vecs(c->tree.n), A;
    for (int z = 0; z < c->tree.n; ++z) {
        if (!c->tree.leaf(z)) continue;
        const cplx* p = (const cplx*)(leaf_vecs + leaf_offsets[z]);
        vecs[z].assign(p, p + c->tree.phys[z]);
        double nrm = 0;
        for (auto& v : vecs[z]) nrm += std::norm(v);
        if (!(nrm > 0) || !std::isfinite(nrm)) return fail(c, TTN_E_INVALID, "leaf vector " + std::to_string(z) + " is zero or not finite");
    }
    ttn::product_state(c->tree, vecs, A);
    return take_state(c, A);
}

// Shared by the single- and multi-set Hamiltonian setters.  A Hamiltonian
// with another set count than the state's converts a single-set state into
// a multi-set one: set 0 is the old state, every other set starts empty
// (copies of set 0's isometries with a zero top tensor).
static ttn_status set_ham(ttn_ctx* c, int n_sets, int n_terms, const ttn_c128* coeff, const int* term_ptr,
                          const int* factor_leaf, const ttn_c128* factor_mats, const int64_t* factor_mat_off,
                          const int* bra, const int* ket, int hermitian) {
    ttn_status u = usable(c); if (u) return u;
    if (n_terms > 0 && term_ptr && term_ptr[n_terms] > 0 && (!factor_leaf || !factor_mats || !factor_mat_off))
        return fail(c, TTN_E_INVALID, "null factor arrays");
    ttn::Hamiltonian h;
    std::string msg = ttn::build_hamiltonian(c->tree, n_terms, (const cplx*)coeff, term_ptr, factor_leaf,
                                             (const cplx*)factor_mats, factor_mat_off, hermitian, h, n_sets, bra,
                                             ket);
    if (!msg.empty()) return fail(c, TTN_E_INVALID, msg);
    const int old_sets = c->plan.nset;
    if (old_sets != n_sets && old_sets != 1)
        return fail(c, TTN_E_INVALID, "the state has " + std::to_string(old_sets) + " sets, the operator " +
                    std::to_string(n_sets));
    ttn::Plan P;
    msg = ttn::make_plan(c->tree, &h, c->precision, P);
    if (!msg.empty()) return fail(c, TTN_E_INVALID, msg);
    // a single-set state becoming multi-set
    std::vector<std::vector<cplx>> A;
    const bool convert = old_sets != n_sets;
    if (convert) {
        if (c->resident) {
            ttn_status s = download_state(c, A);
            if (s) return s;
        } else {
            A = c->host_A;
        }
        for (int z = 0; z < c->tree.n; ++z) {
            const int64_t sz = c->tree.size[z];
            std::vector<cplx> blk(A[z].begin(), A[z].begin() + sz);
            A[z].resize((size_t)n_sets * sz);
            for (int a = 1; a < n_sets; ++a)
                for (int64_t i = 0; i < sz; ++i) A[z][a * sz + i] = z == 0 ? cplx(0.0) : blk[i];
        }
    }
    {
        const int nf = n_terms > 0 && term_ptr ? term_ptr[n_terms] : 0;
        int64_t nm = 0;
        for (int f = 0; f < nf; ++f) {
            const int64_t d = c->tree.phys[factor_leaf[f]];
            nm = std::max<int64_t>(nm, factor_mat_off[f] + d * d);
        }
        std::vector<cplx> sc((const cplx*)coeff, (const cplx*)coeff + n_terms);
        std::vector<int> sp(term_ptr, term_ptr + (n_terms > 0 ? n_terms + 1 : 0));
        std::vector<int> sl(factor_leaf ? factor_leaf : sp.data(), factor_leaf ? factor_leaf + nf : sp.data());
        std::vector<cplx> sm_((const cplx*)factor_mats, (const cplx*)factor_mats + (nf > 0 ? nm : 0));
        std::vector<int64_t> so(factor_mat_off ? factor_mat_off : nullptr, factor_mat_off ? factor_mat_off + nf : nullptr);
        c->sop_coeff.swap(sc); c->sop_ptr.swap(sp); c->sop_leaf.swap(sl);
        c->sop_mats.swap(sm_); c->sop_off.swap(so);
        c->sop_herm = hermitian;
        c->sop_nsets = n_sets;
        c->sop_bra.assign(bra && n_sets > 1 ? bra : nullptr, bra && n_sets > 1 ? bra + n_terms : nullptr);
        c->sop_ket.assign(ket && n_sets > 1 ? ket : nullptr, ket && n_sets > 1 ? ket + n_terms : nullptr);
    }
    if (!c->resident) {
        c->ham = h;
        c->has_h = true;
        c->plan = P;
        if (convert) c->host_A.swap(A);
        return TTN_OK;
    }
    if (convert) {
        char* fresh = nullptr;
        cudaError_t ae = dev_alloc(c, &fresh, P.total_bytes);
        if (ae != cudaSuccess) return alloc_fail(c, ae, "device allocation (state)");
        dev_free(c, c->d_state);
        c->d_state = fresh;
        c->state_bytes = P.total_bytes;
        CK(cudaMemsetAsync(c->d_state, 0, c->state_bytes, c->stream), "memset");
    } else if ((size_t)P.total_bytes > c->state_bytes) {
        char* fresh = nullptr;
        cudaError_t ae = dev_alloc(c, &fresh, P.total_bytes);
        if (ae != cudaSuccess) return alloc_fail(c, ae, "device allocation (state)");
        CK(cudaMemsetAsync(fresh, 0, P.total_bytes, c->stream), "memset");
        CK(cudaMemcpyAsync(fresh, c->d_state, P.bond_off, cudaMemcpyDeviceToDevice, c->stream), "state copy");
        CK(cudaStreamSynchronize(c->stream), "stream synchronize");
        dev_free(c, c->d_state);
        c->d_state = fresh;
        c->state_bytes = P.total_bytes;
    }
    c->ham = h;
    c->has_h = true;
    c->plan = P;
    ttn_status s = upload_ops(c);
    if (s) { c->failed = true; return s; }
    if (convert) {
        s = upload_state(c, A);
        if (s) { c->failed = true; return s; }
    }
    return run_program(c, c->init_p, 0.0, 1);
}

ttn_status ttn_set_sop_hamiltonian(ttn_ctx* c, int n_terms, const ttn_c128* coeff, const int* term_ptr,
                                   const int* factor_leaf, const ttn_c128* factor_mats,
                                   const int64_t* factor_mat_off, int hermitian) {
    if (c && c->plan.nset > 1)
        return fail(c, TTN_E_INVALID, "the state is multi-set: use ttn_set_multiset_hamiltonian");
    return set_ham(c, 1, n_terms, coeff, term_ptr, factor_leaf, factor_mats, factor_mat_off, nullptr, nullptr,
                   hermitian);
}

ttn_status ttn_set_multiset_hamiltonian(ttn_ctx* c, int n_sets, int n_terms, const ttn_c128* coeff,
                                        const int* term_ptr, const int* factor_leaf, const ttn_c128* factor_mats,
                                        const int64_t* factor_mat_off, const int* bra, const int* ket,
                                        int hermitian) {
    if (!c) return TTN_E_INVALID;
    if (n_sets < 1 || n_sets > TTN_MAX_SETS) return fail(c, TTN_E_INVALID, "n_sets must be in 1.." + std::to_string(TTN_MAX_SETS));
    if (n_terms > 0 && (!bra || !ket)) return fail(c, TTN_E_INVALID, "null bra / ket set indices");
    return set_ham(c, n_sets, n_terms, coeff, term_ptr, factor_leaf, factor_mats, factor_mat_off, bra, ket,
                   hermitian);
}

ttn_status ttn_set_multiset_state(ttn_ctx* c, int n_sets, const ttn_c128* tensors, const int64_t* offsets) {
    ttn_status u = usable(c); if (u) return u;
    if (!tensors || !offsets) return fail(c, TTN_E_INVALID, "null tensors / offsets");
    if (n_sets != c->plan.nset)
        return fail(c, TTN_E_INVALID, "n_sets must equal the set count of the multi-set Hamiltonian (" +
                    std::to_string(c->plan.nset) + ")");
    const int n = c->tree.n;
    std::vector<std::vector<cplx>> A(n);
    for (int z = 0; z < n; ++z) A[z].resize((size_t)n_sets * c->tree.size[z]);
    for (int a = 0; a < n_sets; ++a)
        for (int z = 0; z < n; ++z) {
            const int64_t i = (int64_t)a * n + z;
            if (offsets[i + 1] - offsets[i] != c->tree.size[z])
                return fail(c, TTN_E_INVALID, "tensor of set " + std::to_string(a) + ", node " + std::to_string(z) +
                            " has the wrong size");
            const cplx* p = (const cplx*)(tensors + offsets[i]);
            for (int64_t q = 0; q < c->tree.size[z]; ++q) {
                if (!std::isfinite(p[q].real()) || !std::isfinite(p[q].imag()))
                    return fail(c, TTN_E_INVALID, "non-finite tensor entry");
                A[z][a * c->tree.size[z] + q] = p[q];
            }
        }
    return take_state(c, A);
}

ttn_status ttn_get_multiset_state(ttn_ctx* c, int alpha, ttn_c128* tensors, int64_t* offsets) {
    if (!c || !tensors || !offsets) return TTN_E_INVALID;
    if (alpha < 0 || alpha >= c->plan.nset) return fail(c, TTN_E_INVALID, "alpha outside the sets");
    std::vector<std::vector<cplx>> A;
    if (c->resident) {
        cudaSetDevice(c->device);
        ttn_status s = download_state(c, A);
        if (s) return s;
    }
    const auto& src = c->resident ? A : c->host_A;
    int64_t o = 0;
    for (int z = 0; z < c->tree.n; ++z) {
        offsets[z] = o;
        std::memcpy(tensors + o, src[z].data() + (size_t)alpha * c->tree.size[z], c->tree.size[z] * 16);
        o += c->tree.size[z];
    }
    offsets[c->tree.n] = o;
    return TTN_OK;
}

ttn_status ttn_set_populations(ttn_ctx* c, double* pops) {
    ttn_status u = ready(c); if (u) return u;
    if (!pops) return fail(c, TTN_E_INVALID, "pops is NULL");
    const int S = c->plan.nset;
    if (S == 1) {
        ttn_status s = ttn_norm_energy(c, &pops[0], nullptr);
        return s;
    }
    ttn_status s = run_program(c, c->setpop_p, 0.0, 1);
    if (s) return s;
    std::vector<double> sc(2 * (size_t)S);
    CK(cudaMemcpyAsync(sc.data(), c->d_state + c->plan.setpop_off, sc.size() * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream), "scalar copy");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    for (int a = 0; a < S; ++a) pops[a] = sc[2 * a];
    return TTN_OK;
}

ttn_status ttn_n_sets(const ttn_ctx* c, int* n_sets) {
    if (!c || !n_sets) return TTN_E_INVALID;
    *n_sets = c->plan.nset;
    return TTN_OK;
}

ttn_status ttn_save(ttn_ctx* c, void* buf, size_t* len) {
    ttn_status u = usable(c); if (u) return u;
    if (!len) return fail(c, TTN_E_INVALID, "len is NULL");
    const bool sets = c->plan.nset > 1;
    std::vector<std::vector<cplx>> A;
    int64_t steps = c->saved_steps;
    double flops[2] = {c->saved_flops, c->saved_flops64};
    if (c->resident) {
        ttn_status s = download_state(c, A);
        if (s) return s;
        int st = 0;
        CK(cudaMemcpyAsync(&st, c->d_state + c->plan.steps_off, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "counter copy");
        CK(cudaMemcpyAsync(flops, c->d_state + c->plan.flops_off, sizeof(flops), cudaMemcpyDeviceToHost, c->stream), "counter copy");
        CK(cudaStreamSynchronize(c->stream), "stream synchronize");
        steps = st;
    } else {
        A = c->host_A;
    }
    Writer w;
    w.put<uint32_t>(sets ? kCkptMagicSets : kCkptMagic);
    w.put<int32_t>(c->precision);
    w.put_vec(c->tree.parent);
    w.put_vec(c->tree.phys);
    std::vector<int> bond(c->tree.n);
    for (int z = 0; z < c->tree.n; ++z) bond[z] = z == 0 ? 1 : c->tree.bond[z];
    w.put_vec(bond);
    w.put<int64_t>(steps);
    w.put<double>(flops[0]);
    w.put<double>(flops[1]);
    w.put<int32_t>(c->has_h ? 1 : 0);
    w.put<int32_t>(c->sop_herm);
    w.put_vec(c->sop_coeff);
    w.put_vec(c->sop_ptr);
    w.put_vec(c->sop_leaf);
    w.put_vec(c->sop_off);
    w.put_vec(c->sop_mats);
    if (sets) {
        w.put<int32_t>(c->sop_nsets);
        w.put_vec(c->sop_bra);
        w.put_vec(c->sop_ket);
    }
    for (int z = 0; z < c->tree.n; ++z) w.put_vec(A[z]);
    const size_t need = w.b.size();
    if (!buf) { *len = need; return TTN_OK; }
    if (*len < need) { *len = need; return fail(c, TTN_E_INVALID, "buffer too small for the checkpoint"); }
    std::memcpy(buf, w.b.data(), need);
    *len = need;
    return TTN_OK;
}

ttn_status ttn_load(ttn_ctx* c, const void* buf, size_t len) {
    ttn_status u = usable(c); if (u) return u;
    if (!buf) return fail(c, TTN_E_INVALID, "buf is NULL");
    Reader r{(const char*)buf, len};
    const int64_t big = (int64_t)1 << 40;
    const uint32_t magic = r.get<uint32_t>();
    if ((magic != kCkptMagic && magic != kCkptMagicSets) || !r.ok)
        return fail(c, TTN_E_INVALID, "not a libttn checkpoint");
    r.get<int32_t>();                                // precision of the saving context (informational)
    std::vector<int> parent = r.get_vec<int>(65535), phys = r.get_vec<int>(65535), bond = r.get_vec<int>(65535);
    const int64_t steps = r.get<int64_t>();
    const double f0 = r.get<double>(), f1 = r.get<double>();
    const int has_h = r.get<int32_t>(), herm = r.get<int32_t>();
    std::vector<cplx> coeff = r.get_vec<cplx>(big);
    std::vector<int> ptr = r.get_vec<int>(big), leaf = r.get_vec<int>(big);
    std::vector<int64_t> off = r.get_vec<int64_t>(big);
    std::vector<cplx> mats = r.get_vec<cplx>(big);
    int nsets = 1;
    std::vector<int> bra, ket;
    if (magic == kCkptMagicSets) {
        nsets = r.get<int32_t>();
        bra = r.get_vec<int>(big);
        ket = r.get_vec<int>(big);
        if (r.ok && (nsets < 2 || nsets > TTN_MAX_SETS || !has_h || bra.size() != coeff.size() ||
                     ket.size() != coeff.size()))
            return fail(c, TTN_E_INVALID, "inconsistent multi-set checkpoint");
    }
    if (!r.ok || parent.size() != phys.size() || parent.size() != bond.size() || parent.empty())
        return fail(c, TTN_E_INVALID, "truncated or inconsistent checkpoint");
    ttn::Tree t;
    std::string msg = ttn::build_tree((int)parent.size(), parent.data(), phys.data(), bond.data(), t);
    if (!msg.empty()) return fail(c, TTN_E_INVALID, "checkpoint tree: " + msg);
    std::vector<std::vector<cplx>> A(t.n);
    for (int z = 0; z < t.n; ++z) {
        A[z] = r.get_vec<cplx>(big);
        if (!r.ok || (int64_t)A[z].size() != nsets * t.size[z])
            return fail(c, TTN_E_INVALID, "checkpoint tensor " + std::to_string(z) + " has the wrong size");
    }
    ttn::Hamiltonian h;
    ttn::Plan probe;                                 // plan now, so nothing fails after ctx is modified
    if (has_h) {
        const int nt = (int)coeff.size();
        if ((int)ptr.size() != nt + 1 || ptr[nt] != (int)leaf.size() || leaf.size() != off.size())
            return fail(c, TTN_E_INVALID, "inconsistent Hamiltonian in the checkpoint");
        msg = ttn::build_hamiltonian(t, nt, coeff.data(), ptr.data(), leaf.empty() ? nullptr : leaf.data(),
                                     mats.empty() ? nullptr : mats.data(), off.empty() ? nullptr : off.data(), herm, h,
                                     nsets, bra.empty() ? nullptr : bra.data(), ket.empty() ? nullptr : ket.data());
        if (!msg.empty()) return fail(c, TTN_E_INVALID, "checkpoint Hamiltonian: " + msg);
        msg = ttn::make_plan(t, &h, c->precision, probe);
        if (!msg.empty()) return fail(c, TTN_E_INVALID, "checkpoint Hamiltonian: " + msg);
    }
    // everything validated: replace the context's contents, keeping its residency
    const bool was_resident = c->resident;
    if (c->resident) {
        free_ops(c);
        dev_free(c, c->d_state);
        c->d_state = nullptr;
        c->state_bytes = 0;
        if (c->d_batch) cudaFree(c->d_batch);
        c->d_batch = nullptr;
        c->batch_cap = 0;
        c->resident = false;
    }
    c->tree = t;
    c->has_h = false;
    c->ham = ttn::Hamiltonian();
    ttn::make_plan(c->tree, nullptr, c->precision, c->plan);
    c->host_A.swap(A);
    c->saved_steps = steps;
    c->saved_flops = f0;
    c->saved_flops64 = f1;
    c->sop_coeff.clear(); c->sop_ptr.clear(); c->sop_leaf.clear(); c->sop_off.clear(); c->sop_mats.clear();
    c->sop_nsets = 1; c->sop_bra.clear(); c->sop_ket.clear();
    if (nsets > 1) {
        // the set blocks are restored as saved: the multi-set plan and
        // operator directly, no conversion of a single-set state
        c->plan = probe;
        c->ham = h;
        c->has_h = true;
        c->sop_coeff = coeff; c->sop_ptr = ptr; c->sop_leaf = leaf; c->sop_off = off; c->sop_mats = mats;
        c->sop_herm = herm;
        c->sop_nsets = nsets; c->sop_bra = bra; c->sop_ket = ket;
    } else if (has_h) {
        ttn_status s = ttn_set_sop_hamiltonian(c, (int)coeff.size(), (const ttn_c128*)coeff.data(), ptr.data(),
                                               leaf.empty() ? nullptr : leaf.data(),
                                               mats.empty() ? nullptr : (const ttn_c128*)mats.data(),
                                               off.empty() ? nullptr : off.data(), herm);
        if (s) return s;
    }
    if (was_resident) return ready(c);
    return TTN_OK;
}

ttn_status ttn_set_coefficients(ttn_ctx* c, int n_terms, const ttn_c128* coeff) {
    ttn_status u = usable(c); if (u) return u;
    if (!c->has_h) return fail(c, TTN_E_STATE, "no Hamiltonian set");
    if (n_terms != (int)c->sop_coeff.size() || (n_terms > 0 && !coeff))
        return fail(c, TTN_E_INVALID, "n_terms differs from the Hamiltonian's term count");
    for (int r = 0; r < n_terms; ++r)
        if (!std::isfinite(coeff[r].re) || !std::isfinite(coeff[r].im)) return fail(c, TTN_E_INVALID, "non-finite coefficient");
    // replay the set-up with the stored factors (local copies: the call replaces them)
    const std::vector<int> ptr = c->sop_ptr, leaf = c->sop_leaf, bra = c->sop_bra, ket = c->sop_ket;
    const std::vector<cplx> mats = c->sop_mats;
    const std::vector<int64_t> off = c->sop_off;
    return set_ham(c, c->sop_nsets, n_terms, coeff, ptr.empty() ? nullptr : ptr.data(),
                   leaf.empty() ? nullptr : leaf.data(), mats.empty() ? nullptr : (const ttn_c128*)mats.data(),
                   off.empty() ? nullptr : off.data(), bra.empty() ? nullptr : bra.data(),
                   ket.empty() ? nullptr : ket.data(), c->sop_herm);
}

ttn_status ttn_step(ttn_ctx* c, double dt, int nsteps, const ttn_step_opts* opts) {
    ttn_status u = usable(c); if (u) return u;
    if (!c->has_h) return fail(c, TTN_E_STATE, "no Hamiltonian set");
    u = ready(c); if (u) return u;
    if (nsteps < 0 || !std::isfinite(dt)) return fail(c, TTN_E_INVALID, "bad dt / nsteps");
    if (opts) {
        if (opts->krylov_maxdim > TTN_KMAX) return fail(c, TTN_E_INVALID, "krylov_maxdim must be <= 32");
        if (opts->expand && (!(opts->eps_spawn > 0.0) || opts->chi_max < 1 || opts->chi_max > TTN_MAXCHI))
            return fail(c, TTN_E_INVALID, "expansion needs eps_spawn > 0 and 1 <= chi_max <= 64");
        c->ktol = opts->krylov_tol;
        c->qtol = opts->qr_rank_tol;
        c->kmax = opts->krylov_maxdim > 0 ? opts->krylov_maxdim : TTN_KMAX;
    }
    if (!opts || !opts->expand) return run_program(c, c->step_p, dt, nsteps);
    for (int i = 0; i < nsteps; ++i) {
        ttn_status s = expand_pass(c, dt, opts->eps_spawn, opts->chi_max);
        if (s) return s;
        s = run_program(c, c->step_p, dt, 1);
        if (s) return s;
    }
    return TTN_OK;
}

ttn_status ttn_ground_state(ttn_ctx* c, int nsweeps, double* energies) {
    ttn_status u = usable(c); if (u) return u;
    if (!c->has_h) return fail(c, TTN_E_STATE, "no Hamiltonian set");
    if (!c->ham.hermitian) return fail(c, TTN_E_INVALID, "ground-state sweeps need a Hermitian Hamiltonian");
    if (c->plan.nset > 1) return fail(c, TTN_E_INVALID, "ground-state sweeps are for single-set states");
    if (nsweeps < 0) return fail(c, TTN_E_INVALID, "nsweeps must be >= 0");
    u = ready(c); if (u) return u;
    for (int i = 0; i < nsweeps; ++i) {
        ttn_status s = run_program(c, c->ground_p, 0.0, 1);
        if (s) return s;
        if (energies) {
            CK(cudaMemcpyAsync(&energies[i], c->d_state + c->plan.scal_off + 64, sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream), "energy copy");
            CK(cudaStreamSynchronize(c->stream), "stream synchronize");
            energies[i] += c->plan.e_shift;
        }
    }
    return TTN_OK;
}

ttn_status ttn_step_batch(ttn_ctx* const* ctxs, int n, double dt, int nsteps, const ttn_step_opts* opts) {
    if (!ctxs || n <= 0) return TTN_E_INVALID;
    ttn_ctx* c = ctxs[0];
    for (int i = 0; i < n; ++i) {
        ttn_status u = usable(ctxs[i]); if (u) return u;
        if (!ctxs[i]->has_h) return fail(ctxs[i], TTN_E_STATE, "no Hamiltonian set");
        u = ready(ctxs[i]); if (u) return u;
        if (ctxs[i]->precision != c->precision) return fail(c, TTN_E_INVALID, "mixed precisions in one batch");
        if (opts) {
            if (opts->expand) return fail(c, TTN_E_INVALID, "subspace expansion is run per context: use ttn_step");
            ctxs[i]->ktol = opts->krylov_tol;
            ctxs[i]->qtol = opts->qr_rank_tol;
            ctxs[i]->kmax = opts->krylov_maxdim > 0 ? std::min(opts->krylov_maxdim, TTN_KMAX) : TTN_KMAX;
        }
    }
    if (c->batch_cap < n) {
        if (c->d_batch) cudaFree(c->d_batch);
        c->d_batch = nullptr;
        CK(cudaMalloc(&c->d_batch, sizeof(TtnInstance) * n), "cudaMalloc (batch)");
        c->batch_cap = n;
    }
    std::vector<TtnInstance> ins(n);
    for (int i = 0; i < n; ++i) ins[i] = make_instance(ctxs[i], ctxs[i]->step_p);
    // one launch: every instance gets the largest team any of them asks
    // for (automatic choice in a batch: one block each unless a dimension
    // needs a cluster)
    int cluster = 1;
    for (int i = 0; i < n; ++i) {
        const int need = ctxs[i]->plan.max_chi > ttn::kSoloMaxDim ? 2 : 1;
        cluster = std::max(cluster, ctxs[i]->cluster_req > 0 ? std::max(ctxs[i]->cluster_req, need) : need);
    }
    CK(cudaMemcpyAsync(c->d_batch, ins.data(), sizeof(TtnInstance) * n, cudaMemcpyHostToDevice, c->stream), "batch upload");
    bool tc = false;
    for (int i = 0; i < n; ++i) tc |= ttn::ctx_uses_tc(ctxs[i]);
    int e = ttn_launch_program(c->precision, cluster, c->d_batch, n, dt, nsteps, c->stream, tc);
    if (e != 0) return cuda_fail(c, (cudaError_t)e, "kernel launch");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    for (int i = 0; i < n; ++i) {
        ctxs[i]->stream = ctxs[i]->stream;
        ttn_status s = check_status(ctxs[i]);
        if (s) return s;
    }
    return TTN_OK;
}

ttn_status ttn_norm_energy(ttn_ctx* c, double* norm2, ttn_c128* energy) {
    ttn_status u = ready(c); if (u) return u;
    ttn_status s = run_program(c, c->ne_p, 0.0, 1);
    if (s) return s;
    double sc[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(sc, c->d_state + c->plan.scal_off, sizeof(sc), cudaMemcpyDeviceToHost, c->stream), "scalar copy");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    if (norm2) *norm2 = sc[0];
    if (energy) {
        if (!c->has_h) return fail(c, TTN_E_STATE, "no Hamiltonian set");
        energy->re = sc[2] / sc[0] + c->plan.e_shift;     // the bulk works with H - e_shift
        energy->im = sc[3] / sc[0];
    }
    return TTN_OK;
}

ttn_status ttn_reduced_density(ttn_ctx* c, int leaf, ttn_c128* out) {
    ttn_status u = ready(c); if (u) return u;
    if (c->plan.nset > 1) return fail(c, TTN_E_INVALID, "leaf densities are for single-set states: use ttn_set_populations");
    if (leaf < 0 || leaf >= c->tree.n || !c->tree.leaf(leaf) || !out) return fail(c, TTN_E_INVALID, "leaf must be a leaf node");
    ttn_status s = run_program(c, c->rdm_p[leaf], 0.0, 1);
    if (s) return s;
    double nrm = 0;
    s = ttn_norm_energy(c, &nrm, nullptr);
    if (s) return s;
    int d = c->tree.phys[leaf];
    const ttn::SlotInfo& sl = c->plan.slots[c->plan.rdm_slot[leaf]];
    std::vector<char> raw(d * d * c->plan.esz);
    CK(cudaMemcpyAsync(raw.data(), c->d_ops + sl.off, raw.size(), cudaMemcpyDeviceToHost, c->stream), "rdm copy");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    std::vector<cplx> g(d * d);
    from_bulk(raw.data(), d * d, c->plan.esz, g.data());
    // the device computes conj(rho) * <Psi|Psi>
    for (int i = 0; i < d * d; ++i) {
        cplx v = std::conj(g[i]) / nrm;
        out[i].re = v.real(); out[i].im = v.imag();
    }
    return TTN_OK;
}

ttn_status ttn_expect(ttn_ctx* c, int n_obs, const int* leaf, const ttn_c128* ops, const int64_t* op_off, ttn_c128* out) {
    ttn_status u = usable(c); if (u) return u;
    if (n_obs < 0 || (n_obs > 0 && (!leaf || !ops || !op_off || !out))) return fail(c, TTN_E_INVALID, "bad arguments");
    for (int i = 0; i < n_obs; ++i) {
        int l = leaf[i];
        if (l < 0 || l >= c->tree.n || !c->tree.leaf(l)) return fail(c, TTN_E_INVALID, "leaf must be a leaf node");
        int d = c->tree.phys[l];
        std::vector<ttn_c128> rho(d * d);
        ttn_status s = ttn_reduced_density(c, l, rho.data());
        if (s) return s;
        cplx acc = 0;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                cplx o(ops[op_off[i] + b * d + a].re, ops[op_off[i] + b * d + a].im);
                acc += cplx(rho[a * d + b].re, rho[a * d + b].im) * o;
            }
        out[i].re = acc.real(); out[i].im = acc.imag();
    }
    return TTN_OK;
}

ttn_status ttn_vacuum_projection(ttn_ctx* c, int keep_leaf, ttn_c128* out) {
    ttn_status u = ready(c); if (u) return u;
    if (c->plan.nset > 1) return fail(c, TTN_E_INVALID, "vacuum projections are for single-set states");
    if (keep_leaf < 0 || keep_leaf >= c->tree.n || !c->tree.leaf(keep_leaf) || !out) return fail(c, TTN_E_INVALID, "keep_leaf must be a leaf");
    ttn_status s = run_program(c, c->vac_p[keep_leaf], 0.0, 1);
    if (s) return s;
    int d = c->tree.phys[keep_leaf];
    const ttn::SlotInfo& sl = c->plan.slots[c->plan.vac_slot[keep_leaf]];
    std::vector<char> raw(d * c->plan.esz);
    CK(cudaMemcpyAsync(raw.data(), c->d_ops + sl.off, raw.size(), cudaMemcpyDeviceToHost, c->stream), "vector copy");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    from_bulk(raw.data(), d, c->plan.esz, (cplx*)out);
    return TTN_OK;
}

ttn_status ttn_get_state(ttn_ctx* c, ttn_c128* tensors, int64_t* offsets) {
    if (!c || !tensors || !offsets) return TTN_E_INVALID;
    if (c->plan.nset > 1) return fail(c, TTN_E_INVALID, "the state is multi-set: use ttn_get_multiset_state");
    std::vector<std::vector<cplx>> A;
    if (c->resident) {
        cudaSetDevice(c->device);
        ttn_status s = download_state(c, A);
        if (s) return s;
    }
    const auto& src = c->resident ? A : c->host_A;
    int64_t o = 0;
    for (int z = 0; z < c->tree.n; ++z) {
        offsets[z] = o;
        std::memcpy(tensors + o, src[z].data(), c->tree.size[z] * 16);
        o += c->tree.size[z];
    }
    offsets[c->tree.n] = o;
    return TTN_OK;
}

ttn_status ttn_tree(const ttn_ctx* c, int* n_nodes, int* parent, int* phys_dim, int* bond_dim) {
    if (!c || !n_nodes) return TTN_E_INVALID;
    *n_nodes = c->tree.n;
    for (int z = 0; z < c->tree.n; ++z) {
        if (parent) parent[z] = c->tree.parent[z];
        if (phys_dim) phys_dim[z] = c->tree.phys[z];
        if (bond_dim) bond_dim[z] = z == 0 ? 1 : c->tree.bond[z];
    }
    return TTN_OK;
}

ttn_status ttn_bond_dims(ttn_ctx* c, int* out) {
    if (!c || !out) return TTN_E_INVALID;
    for (int z = 0; z < c->tree.n; ++z) out[z] = z == 0 ? 1 : c->tree.bond[z];
    return TTN_OK;
}

namespace {

// Validate a kernel-level operator and build its entry / slot tables.
ttn_status build_heff_tables(int D, const int* dims, int n_terms, const ttn_c128* coeff, const int* factor,
                             int n_mats, const void* const* mats, int64_t* S_out, std::vector<TtnEntry>& ents,
                             std::vector<TtnSlot>& slots) {
    if (D < 1 || D > TTN_MAXD || !dims || n_terms < 0 || (n_terms > 0 && (!coeff || !factor)) || n_mats < 0 ||
        (n_mats > 0 && !mats))
        return fail(nullptr, TTN_E_INVALID, "bad operator description");
    int64_t S = 1;
    for (int j = 0; j < D; ++j) {
        if (dims[j] < 1 || dims[j] > TTN_MAXCHI) return fail(nullptr, TTN_E_INVALID, "dims out of range");
        S *= dims[j];
    }
    slots.assign(std::max(1, n_mats), TtnSlot{nullptr, 0, 0});
    for (int i = 0; i < n_mats; ++i) {
        if (!mats[i]) return fail(nullptr, TTN_E_INVALID, "null matrix pointer");
        slots[i].ptr = const_cast<void*>(mats[i]);
    }
    ents.clear();
    for (int t = 0; t < n_terms; ++t) {
        TtnEntry e{};
        e.wr = coeff[t].re; e.wi = coeff[t].im; e.out = -1;
        for (int j = 0; j < TTN_MAXD; ++j) e.slot[j] = -1;
        for (int j = 0; j < D; ++j) {
            int f = factor[t * D + j];
            if (f < -1 || f >= n_mats) return fail(nullptr, TTN_E_INVALID, "factor index out of range");
            e.slot[j] = f;
            if (f >= 0) {
                if (slots[f].rows && slots[f].rows != dims[j]) return fail(nullptr, TTN_E_INVALID, "matrix used on indices of different dimension");
                slots[f].rows = slots[f].cols = dims[j];
            }
        }
        ents.push_back(e);
    }
    // adjacent entries sharing their last factor are summed before it is applied
    auto last = [D](const TtnEntry& e) {
        int lm = -1;
        for (int j = 0; j < D; ++j) if (e.slot[j] >= 0) lm = j;
        return std::make_pair(lm, lm >= 0 ? e.slot[lm] : -1);
    };
    std::stable_sort(ents.begin(), ents.end(), [&](const TtnEntry& a, const TtnEntry& b) { return last(a) < last(b); });
    *S_out = S;
    return TTN_OK;
}

}  // namespace

ttn_status ttn_heff_apply(void* stream, int D, const int* dims, int n_terms, const ttn_c128* coeff, const int* factor,
                          int n_mats, const void* const* mats, const ttn_c128* x, ttn_c128* y) {
    std::vector<TtnEntry> ents;
    std::vector<TtnSlot> slots;
    int64_t S = 0;
    ttn_status st = build_heff_tables(D, dims, n_terms, coeff, factor, n_mats, mats, &S, ents, slots);
    if (st) return st;
    if (!x || !y) return fail(nullptr, TTN_E_INVALID, "null tensor pointer");
    cudaStream_t s = (cudaStream_t)stream;
    ttn_ctx* c = nullptr;   // errors of this call are reported through ttn_last_error(NULL)
    const size_t tens = (size_t)S * 16;
    const size_t eb = std::max<size_t>(1, ents.size()) * sizeof(TtnEntry), sb = slots.size() * sizeof(TtnSlot);
    char* scratch = nullptr;
    CK(cudaMalloc(&scratch, 3 * tens + eb + sb), "cudaMalloc (scratch)");
    char* de = scratch + 3 * tens;
    char* ds = de + eb;
    cudaError_t e = cudaMemcpyAsync(de, ents.data(), ents.size() * sizeof(TtnEntry), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ds, slots.data(), sb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = (cudaError_t)ttn_launch_heff((const TtnEntry*)de, (int)ents.size(), (const TtnSlot*)ds, D, dims, x, y,
                                         scratch, scratch + tens, scratch + 2 * tens, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (e != cudaSuccess) return cuda_fail(c, e, "ttn_heff_apply");
    return TTN_OK;
}

ttn_status ttn_heff_apply_noalloc(void* stream, int D, const int* dims, int n_terms, const ttn_c128* coeff,
                                  const int* factor, int n_mats, const void* const* mats, const ttn_c128* x,
                                  ttn_c128* y) {
    std::vector<TtnEntry> ents;
    std::vector<TtnSlot> slots;
    int64_t S = 0;
    ttn_status st = build_heff_tables(D, dims, n_terms, coeff, factor, n_mats, mats, &S, ents, slots);
    if (st) return st;
    if (!x || !y) return fail(nullptr, TTN_E_INVALID, "null tensor pointer");
    if (S > TTN_NOALLOC_MAX_ELEMS)
        return fail(nullptr, TTN_E_INVALID, "tensor has " + std::to_string(S) + " elements; the allocation-free entry point takes at most " +
                                                std::to_string(TTN_NOALLOC_MAX_ELEMS));
    if (n_terms > TTN_NOALLOC_MAX_TERMS || n_mats > TTN_NOALLOC_MAX_MATS)
        return fail(nullptr, TTN_E_INVALID, "at most " + std::to_string(TTN_NOALLOC_MAX_TERMS) + " terms and " +
                                                std::to_string(TTN_NOALLOC_MAX_MATS) + " matrices in the allocation-free entry point");
    cudaStream_t s = (cudaStream_t)stream;
    ttn_ctx* c = nullptr;
    cudaError_t e = (cudaError_t)ttn_launch_heff_noalloc(ents.data(), (int)ents.size(), slots.data(), (int)slots.size(),
                                                         D, dims, x, y, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "ttn_heff_apply_noalloc");
    return TTN_OK;
}

ttn_status ttn_set_cluster(ttn_ctx* c, int blocks) {
    if (!c) return fail(nullptr, TTN_E_INVALID, "ctx is NULL");
    if (blocks < 0 || blocks > TTN_MAX_CLUSTER || (blocks & (blocks - 1)) != 0)
        return fail(c, TTN_E_INVALID, "blocks must be 0 (automatic), 1, 2, 4, 8 or 16");
    c->cluster_req = blocks;
    return TTN_OK;
}

ttn_status ttn_get_cluster(const ttn_ctx* c, int* blocks) {
    if (!c || !blocks) return fail(nullptr, TTN_E_INVALID, "NULL argument");
    *blocks = ttn::ctx_cluster(c);
    return TTN_OK;
}

// Autotuning: time whole steps of the context's own problem for candidate
// launch shapes and mode-product routines, starting every trial from the
// same snapshot of everything a step modifies (state arena: tensors, bond
// buffer, workspace, counters; operator arena: environment and channel
// matrices), and keep the fastest.  The context ends exactly as it began.
ttn_status ttn_autotune(ttn_ctx* c, double dt, int steps, int flags, double* tuned_ms) {
    ttn_status u = usable(c); if (u) return u;
    if (!c->has_h) return fail(c, TTN_E_STATE, "no Hamiltonian set");
    if (steps < 1 || steps > 1000 || !std::isfinite(dt)) return fail(c, TTN_E_INVALID, "need 1 <= steps <= 1000, finite dt");
    u = ready(c); if (u) return u;
    const size_t slot_bytes = ops_layout(c->plan).slot_bytes;
    char *snap_s = nullptr, *snap_o = nullptr;
    cudaError_t ae = dev_alloc(c, &snap_s, c->state_bytes);
    if (ae == cudaSuccess) ae = dev_alloc(c, &snap_o, std::max<size_t>(slot_bytes, 256));
    if (ae != cudaSuccess) { dev_free(c, snap_s); return alloc_fail(c, ae, "autotune snapshot"); }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    ttn_status st = TTN_OK;
    auto restore = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(c->d_state, snap_s, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess && slot_bytes)
            e = cudaMemcpyAsync(c->d_ops, snap_o, slot_bytes, cudaMemcpyDeviceToDevice, c->stream);
        return e;
    };
    auto trial = [&](double* ms) -> ttn_status {
        cudaError_t e = restore();
        TtnInstance in = make_instance(c, c->step_p);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_inst, &in, sizeof(in), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess)
            e = (cudaError_t)ttn_launch_program(c->precision, ttn::ctx_cluster(c), c->d_inst, 1, dt, steps,
                                                c->stream, ttn::ctx_uses_tc(c));
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "autotune launch");
        ttn_status s2 = check_status(c);
        if (s2) return s2;
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        *ms = f;
        c->tune_trials++;
        return TTN_OK;
    };
    do {
        cudaError_t e = cudaMemcpyAsync(snap_s, c->d_state, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess && slot_bytes)
            e = cudaMemcpyAsync(snap_o, c->d_ops, slot_bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) { st = cuda_fail(c, e, "autotune snapshot"); break; }
        c->tune_trials = 0;
        double best = 0.0;
        if ((st = trial(&best))) break;           // the configuration as given
        c->tune_default_ms = best;
        if (flags & 1) {                           // block count
            const int need = c->plan.max_chi > ttn::kSoloMaxDim ? 2 : 1;
            int best_b = c->cluster_req;
            for (int b = need; b <= TTN_MAX_CLUSTER && !st; b *= 2) {
                if (b > 1) {
                    int act = 0;
                    if (ttn_cluster_capacity(c->precision, b, &act) != 0 || act < 1) { cudaGetLastError(); continue; }
                }
                const int keep = c->cluster_req;
                c->cluster_req = b;
                double ms = 0.0;
                st = trial(&ms);
                if (!st && ms < best) { best = ms; best_b = b; }
                c->cluster_req = keep;
            }
            if (st) break;
            c->cluster_req = best_b;
        }
        if (flags & 2) {                           // mode-product routine per dimension, largest first
            std::set<int> dims;
            for (int z = 0; z < c->tree.n; ++z)
                for (int d : c->tree.dims[z]) if (d >= 4) dims.insert(d);
            const int fibre_lim = c->precision == TTN_MIXED ? 32 : 16;
            for (auto it = dims.rbegin(); it != dims.rend() && !st; ++it) {
                const int n = *it;
                std::vector<int> cands;
                if (n <= fibre_lim) cands.push_back(1);                        // staged instead of fibre
                if ((flags & 4) && c->precision == TTN_MIXED && n <= 48) cands.push_back(2);   // tensor cores
                const unsigned char keep = c->mp_variant[n];
                unsigned char best_v = keep;
                for (int v : cands) {
                    c->mp_variant[n] = (unsigned char)v;
                    double ms = 0.0;
                    st = trial(&ms);
                    if (st) break;
                    if (ms < best) { best = ms; best_v = (unsigned char)v; }
                }
                c->mp_variant[n] = best_v;
            }
            if (st) break;
        }
        c->tune_ms = best;
        if (tuned_ms) *tuned_ms = best;
        cudaError_t r = restore();
        if (r == cudaSuccess) r = cudaStreamSynchronize(c->stream);
        if (r != cudaSuccess) st = cuda_fail(c, r, "autotune restore");
    } while (false);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(c->stream);
    dev_free(c, snap_s);
    dev_free(c, snap_o);
    return st;
}

ttn_status ttn_operator_dims(const ttn_ctx* c, int* out) {
    if (!c || !out) return fail(nullptr, TTN_E_INVALID, "NULL argument");
    if (!c->has_h) return fail(nullptr, TTN_E_STATE, "no Hamiltonian set");
    for (int z = 0; z < c->tree.n; ++z)
        out[z] = z < (int)c->plan.op_bond_dim.size() ? c->plan.op_bond_dim[z] : 0;
    return TTN_OK;
}

ttn_status ttn_set_tuning(ttn_ctx* c, int blocks, const unsigned char* variants) {
    if (!c) return fail(nullptr, TTN_E_INVALID, "ctx is NULL");
    if (blocks < 0 || blocks > TTN_MAX_CLUSTER || (blocks & (blocks - 1)) != 0)
        return fail(c, TTN_E_INVALID, "blocks must be 0 (automatic), 1, 2, 4, 8 or 16");
    if (variants)
        for (int n = 0; n <= TTN_MAXCHI; ++n)
            if (variants[n] > 2) return fail(c, TTN_E_INVALID, "mode-product variants are 0, 1 or 2");
    c->cluster_req = blocks;
    if (variants) std::memcpy(c->mp_variant, variants, TTN_MAXCHI + 1);
    return TTN_OK;
}

ttn_status ttn_tuning(const ttn_ctx* c, int* blocks, unsigned char* variants, double* tuned_ms, double* default_ms,
                      int* trials) {
    if (!c) return fail(nullptr, TTN_E_INVALID, "ctx is NULL");
    if (blocks) *blocks = ttn::ctx_cluster(c);
    if (variants) std::memcpy(variants, c->mp_variant, TTN_MAXCHI + 1);
    if (tuned_ms) *tuned_ms = c->tune_ms;
    if (default_ms) *default_ms = c->tune_default_ms;
    if (trials) *trials = c->tune_trials;
    return TTN_OK;
}

ttn_status ttn_mode_product_c64(void* stream, int64_t L, int n, int64_t R, const void* M, const void* x, void* y,
                                double wr, double wi, int accumulate, int tensor_cores) {
    if (L < 1 || R < 1 || n < 1 || n > TTN_MAXCHI || !M || !x || !y)
        return fail(nullptr, TTN_E_INVALID, "need L, R >= 1, 1 <= n <= 64 and device pointers");
    if (tensor_cores && n > 64) return fail(nullptr, TTN_E_INVALID, "tensor-core mode product: n <= 64");
    cudaStream_t s = (cudaStream_t)stream;
    int* d_status = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d_status, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = (cudaError_t)ttn_launch_mode_product(tensor_cores, L, n, R, M, x, y, wr, wi, accumulate, d_status, s);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (d_status) cudaFreeAsync(d_status, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(nullptr, TTN_E_CUDA, std::string("mode product: ") + cudaGetErrorString(e));
    if (st == 5) return fail(nullptr, TTN_E_TIMEOUT, "tensor-core mode product: an MMA did not complete in time");
    return TTN_OK;
}

ttn_status ttn_pipe_peaks(void* stream, double seconds, double* fp32_tflops, double* fp64_tflops) {
    if (!fp32_tflops || !fp64_tflops || !(seconds > 0.0) || seconds > 60.0)
        return fail(nullptr, TTN_E_INVALID, "need output pointers and 0 < seconds <= 60");
    cudaStream_t s = (cudaStream_t)stream;
    // calibrate on a short run, then time one launch of about `seconds` per pipe
    for (int pipe = 0; pipe < 2; ++pipe) {
        auto run = pipe == 0 ? ttn_pipe_peak_fp32 : ttn_pipe_peak_fp64;
        double tf = 0.0, ms = 0.0;
        int iters = pipe == 0 ? (1 << 16) : (1 << 10);
        int e = run(iters, &tf, &ms, s);
        if (e) return fail(nullptr, TTN_E_CUDA, std::string("pipe benchmark: ") + cudaGetErrorString((cudaError_t)e));
        const double scale = std::max(1.0, seconds * 1e3 / std::max(ms, 1e-3));
        iters = (int)std::min(2e9, iters * scale);
        e = run(iters, &tf, &ms, s);
        if (e) return fail(nullptr, TTN_E_CUDA, std::string("pipe benchmark: ") + cudaGetErrorString((cudaError_t)e));
        (pipe == 0 ? *fp32_tflops : *fp64_tflops) = tf;
    }
    return TTN_OK;
}

ttn_status ttn_set_device(int device) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, TTN_E_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return TTN_OK;
}

ttn_status ttn_step_stats(ttn_ctx* c, int64_t* steps_done, double* flops, uint64_t* stamps, int max_stamps,
                          int* n_stamps) {
    if (!c) return TTN_E_INVALID;
    if (!c->resident) {
        if (steps_done) *steps_done = c->saved_steps;
        if (flops) *flops = c->saved_flops;
        if (n_stamps) *n_stamps = 0;
        return TTN_OK;
    }
    cudaSetDevice(c->device);
    int steps = 0;
    double fl = 0.0;
    CK(cudaMemcpyAsync(&steps, c->d_state + c->plan.steps_off, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "stats copy");
    CK(cudaMemcpyAsync(&fl, c->d_state + c->plan.flops_off, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "stats copy");
    std::vector<unsigned long long> raw(c->plan.max_stamps);
    CK(cudaMemcpyAsync(raw.data(), c->d_state + c->plan.stamps_off, raw.size() * 8, cudaMemcpyDeviceToHost, c->stream), "stats copy");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    if (steps_done) *steps_done = steps;
    if (flops) *flops = fl;
    int n = std::min(std::min(max_stamps, steps), c->plan.max_stamps);
    if (n < 0) n = 0;
    if (stamps)
        for (int i = 0; i < n; ++i) {
            int s = steps - n + i;
            stamps[i] = raw[s % c->plan.max_stamps];
        }
    if (n_stamps) *n_stamps = stamps ? n : 0;
    return TTN_OK;
}

ttn_status ttn_flop_counts(ttn_ctx* c, double* total, double* fp64) {
    if (!c) return TTN_E_INVALID;
    double f[2] = {c->saved_flops, c->saved_flops64};
    if (c->resident) {
        cudaSetDevice(c->device);
        CK(cudaMemcpyAsync(f, c->d_state + c->plan.flops_off, sizeof(f), cudaMemcpyDeviceToHost, c->stream), "counter copy");
        CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    }
    if (total) *total = f[0];
    if (fp64) *fp64 = f[1];
    return TTN_OK;
}

ttn_status ttn_op_cycles(ttn_ctx* c, uint64_t* cycles) {
    if (!c || !cycles) return TTN_E_INVALID;
    if (!c->resident) { std::memset(cycles, 0, 32 * 8); return TTN_OK; }
    cudaSetDevice(c->device);
    CK(cudaMemcpyAsync(cycles, c->d_state + c->plan.cycles_off, 32 * 8, cudaMemcpyDeviceToHost, c->stream), "cycles copy");
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    return TTN_OK;
}

ttn_status ttn_set_stream(ttn_ctx* c, void* stream) {
    if (!c) return TTN_E_INVALID;
    c->stream = (cudaStream_t)stream;
    return TTN_OK;
}

ttn_status ttn_device_bytes(const ttn_ctx* c, size_t* bytes) {
    if (!c || !bytes) return TTN_E_INVALID;
    *bytes = c->state_bytes + c->ops_bytes;
    return TTN_OK;
}

const char* ttn_last_error(const ttn_ctx* c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

void ttn_destroy(ttn_ctx* c) {
    if (!c) return;
    if (!c->resident && !c->d_batch) { delete c; return; }
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_ops(c);
    dev_free(c, c->d_state);
    if (c->d_batch) cudaFree(c->d_batch);
    if (c->pooled && c->stream) cudaStreamSynchronize(c->stream);
    delete c;
}

}  // extern "C"
