// Served form: frames from many simulations, continuous batching.
//
// Simulations are opened at creation or later (vd_server_open_sim), each
// admitted only while the resident state of every open simulation fits the
// HBM budget. The simulations opened together form one group, a batch whose
// instances are those simulations; every simulation's labels, centroids and
// links stay resident on the device. Frames are submitted as they arrive
// (device pointers owned by the caller, with their arrival time).
// vd_server_poll runs the scheduler: it retires finished steps in launch
// order (CUDA events), optionally copies the retired frames' change lists to
// the host, and, while fewer than two steps are in flight, admits the oldest
// waiting frame of every idle simulation -- at most one frame per simulation
// per step, at most max_batch simulations, and only while the resident state
// plus the frames in flight fit the budget -- and enqueues one step for them:
// one vd_batch_push_subset per group that has admitted frames. Frames that
// arrive while a step runs join the next step, so the device always has work
// queued. A simulation is in at most one step in flight, so a retired
// simulation's state is stable until the scheduler admits its next frame.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "vd.h"

vd_status vd_batch_gather_counts_async(vd_batch* b, const int* h_sims, int n, int* d_scratch, int* h_pinned_out);
vd_status vd_batch_gather_changes_list_async(vd_batch* b, void* stream, const int* d_insts, const long long* d_off,
                                             int n, long long nb, uint64_t* d_out, uint8_t* d_act);
long long vd_batch_resident_bytes(const vd_batch* b);

namespace {

long long now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// per-instance counts gathered after each step: K, E, n_breaking, n_arising,
// n_matched, error bits, past-frame bubbles, frames finished
constexpr int CNT = 8;

struct Pending {
    long long ticket;
    const float* field;
    long long t_arrival;
    long long t_submit;
    long long bytes;
};

struct Group {
    vd_batch* b = nullptr;
    std::vector<int> sims;   // server ids of its instances
    long long bytes = 0;     // resident device memory
    int open = 0;            // instances not closed
};

struct Sim {
    int group = -1, inst = -1;
    bool open = false, busy = false;
    vd_config cfg;
    std::deque<Pending> q;
};

struct Step {
    cudaEvent_t done = nullptr;
    std::vector<int> sims;           // server ids, group by group
    std::vector<Pending> frames;
    int slot = 0;                    // pinned count buffer
};

// change lists of the frames retired by the last poll, on the host
struct Retired {
    int sim;
    int status;
    int K, n_prev, n_matched, n_edges, nb, na;
    long long frame;
    long long ob, oa, ok;            // offsets into the packed lists
};

}  // namespace

struct vd_server {
    std::vector<Group> groups;
    std::vector<Sim> sims;
    int max_batch = 0;
    long long budget = 0;
    long long inflight_bytes = 0;
    long long next_ticket = 0;
    cudaStream_t s = 0;
    std::deque<Step> flight;
    std::vector<cudaEvent_t> ev_free;
    long long steps = 0, frames_done = 0;
    // two count buffers (one per step in flight): device scratch + pinned host
    int* d_cnt[2] = {nullptr, nullptr};
    int* h_cnt[2] = {nullptr, nullptr};
    int cnt_cap[2] = {0, 0};
    int slot_busy[2] = {0, 0};
    // per-frame change lists (vd_server_keep_changes)
    bool keep = false;
    cudaStream_t cs = nullptr;
    std::unordered_map<long long, Retired> retired;
    unsigned long long* d_chg = nullptr;
    unsigned long long* h_chg = nullptr;
    long long chg_cap = 0, chg_nb = 0;
    unsigned char* d_act = nullptr;
    unsigned char* h_act = nullptr;
    long long act_cap = 0;
    long long* d_off = nullptr;
    long long* h_off = nullptr;
    int* d_ins = nullptr;
    int* h_ins = nullptr;
    int off_cap = 0;
};

namespace {

long long resident(const vd_server* sv) {
    long long r = 0;
    for (const Group& g : sv->groups)
        if (g.b) r += g.bytes;
    return r;
}

// a new group of `n` simulations; their ids are returned in `ids`
vd_status open_group(vd_server* sv, const vd_config* cfgs, int n, int32_t* ids) {
    std::vector<vd_config> c(cfgs, cfgs + n);
    for (vd_config& x : c) x.stream = sv->s;
    Group g;
    vd_status r = vd_batch_create(c.data(), n, &g.b);
    if (r) return r;
    g.bytes = vd_batch_resident_bytes(g.b) + 2ll * (long long)sizeof(int) * (CNT + 1) * n;
    if (resident(sv) + g.bytes > sv->budget) {
        vd_batch_destroy(g.b);
        return VD_ERR_CAPACITY;
    }
    const int gi = (int)sv->groups.size();
    for (int k = 0; k < n; ++k) {
        Sim s;
        s.group = gi;
        s.inst = k;
        s.open = true;
        s.cfg = c[k];
        g.sims.push_back((int)sv->sims.size());
        if (ids) ids[k] = (int32_t)sv->sims.size();
        sv->sims.push_back(std::move(s));
    }
    g.open = n;
    sv->groups.push_back(std::move(g));
    return VD_OK;
}

bool valid_sim(const vd_server* sv, int sim) {
    return sv && sim >= 0 && sim < (int)sv->sims.size() && sv->sims[sim].open;
}

vd_status ensure_cnt(vd_server* sv, int slot, int n) {
    if (sv->cnt_cap[slot] >= n) return VD_OK;
    cudaFree(sv->d_cnt[slot]);
    cudaFreeHost(sv->h_cnt[slot]);
    sv->d_cnt[slot] = nullptr;
    sv->h_cnt[slot] = nullptr;
    sv->cnt_cap[slot] = 0;
    const int cap = std::max(n, 2 * (int)sv->sims.size());
    if (cudaMalloc(&sv->d_cnt[slot], sizeof(int) * (CNT + 1) * cap) != cudaSuccess ||
        cudaMallocHost(&sv->h_cnt[slot], sizeof(int) * CNT * cap) != cudaSuccess)
        return VD_ERR_OOM;
    sv->cnt_cap[slot] = cap;
    return VD_OK;
}

vd_status server_launch(vd_server* sv) {
    // idle simulations with a waiting frame, oldest arrival first
    std::vector<int> cand;
    for (int i = 0; i < (int)sv->sims.size(); ++i)
        if (sv->sims[i].open && !sv->sims[i].busy && !sv->sims[i].q.empty()) cand.push_back(i);
    if (cand.empty()) return VD_OK;
    std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) {
        return sv->sims[a].q.front().t_arrival < sv->sims[b].q.front().t_arrival;
    });
    std::vector<std::vector<int>> per_group(sv->groups.size());
    std::vector<std::vector<Pending>> per_frames(sv->groups.size());
    int taken = 0;
    for (int i : cand) {
        if (taken >= sv->max_batch) break;
        Sim& s = sv->sims[i];
        const Pending& p = s.q.front();
        if (resident(sv) + sv->inflight_bytes + p.bytes > sv->budget) break;   // admission by HBM budget
        sv->inflight_bytes += p.bytes;
        per_group[s.group].push_back(i);
        per_frames[s.group].push_back(p);
        s.q.pop_front();
        s.busy = true;
        ++taken;
    }
    if (!taken) return VD_OK;
    Step st;
    st.slot = sv->slot_busy[0] ? 1 : 0;
    vd_status r = ensure_cnt(sv, st.slot, (int)sv->sims.size());
    if (r) return r;
    sv->slot_busy[st.slot] = 1;
    int base = 0;
    for (size_t gi = 0; gi < per_group.size(); ++gi) {
        if (per_group[gi].empty()) continue;
        Group& g = sv->groups[gi];
        std::vector<int> inst;
        std::vector<const float*> fields;
        for (size_t k = 0; k < per_group[gi].size(); ++k) {
            inst.push_back(sv->sims[per_group[gi][k]].inst);
            fields.push_back(per_frames[gi][k].field);
        }
        r = vd_batch_push_subset(g.b, inst.data(), (int32_t)inst.size(), fields.data());
        if (r) return r;
        r = vd_batch_gather_counts_async(g.b, inst.data(), (int)inst.size(), sv->d_cnt[st.slot] + (CNT + 1) * base,
                                         sv->h_cnt[st.slot] + CNT * base);
        if (r) return r;
        for (size_t k = 0; k < per_group[gi].size(); ++k) {
            st.sims.push_back(per_group[gi][k]);
            st.frames.push_back(per_frames[gi][k]);
        }
        base += (int)inst.size();
    }
    if (sv->ev_free.empty()) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return VD_ERR_CUDA;
        sv->ev_free.push_back(e);
    }
    st.done = sv->ev_free.back();
    sv->ev_free.pop_back();
    if (cudaEventRecord(st.done, sv->s) != cudaSuccess) return VD_ERR_CUDA;
    sv->flight.push_back(std::move(st));
    sv->steps += 1;
    return VD_OK;
}

template <class T>
vd_status grow(T** d, T** h, long long* cap, long long need) {
    if (need <= *cap) return VD_OK;
    cudaFree(*d);
    cudaFreeHost(*h);
    *d = nullptr;
    *h = nullptr;
    *cap = 0;
    const long long c = need + need / 2 + 1024;
    if (cudaMalloc(d, sizeof(T) * c) != cudaSuccess || cudaMallocHost(h, sizeof(T) * c) != cudaSuccess)
        return VD_ERR_OOM;
    *cap = c;
    return VD_OK;
}

// Change lists of the retired frames (whose states no step in flight touches)
// gathered on the side stream and copied to pinned host memory; the lists of
// one group's frames are packed next to each other (one gather per group).
vd_status keep_retired(vd_server* sv, const std::vector<long long>& tickets) {
    std::vector<std::vector<long long>> by_group(sv->groups.size());
    for (long long t : tickets) by_group[sv->sims[sv->retired[t].sim].group].push_back(t);
    long long nb = 0, na = 0, nk = 0;
    for (const std::vector<long long>& ts : by_group)
        for (long long t : ts) {
            Retired& R = sv->retired[t];
            R.ob = nb;
            R.oa = na;
            R.ok = nk;
            if (R.status == VD_OK && R.frame > 0) {
                nb += R.nb;
                na += R.na;
                nk += R.K;
            }
        }
    sv->chg_nb = nb;
    vd_status r = grow(&sv->d_chg, &sv->h_chg, &sv->chg_cap, 2 * nb + na);
    if (!r) r = grow(&sv->d_act, &sv->h_act, &sv->act_cap, nk);
    if (r) return r;
    for (size_t gi = 0; gi < by_group.size(); ++gi) {
        const std::vector<long long>& ts = by_group[gi];
        if (ts.empty()) continue;
        const int n = (int)ts.size();
        if (n + 1 > sv->off_cap) {
            cudaFree(sv->d_off);
            cudaFreeHost(sv->h_off);
            cudaFree(sv->d_ins);
            cudaFreeHost(sv->h_ins);
            sv->off_cap = 0;
            const int c = std::max(n + 1, (int)sv->sims.size() + 1);
            if (cudaMalloc(&sv->d_off, sizeof(long long) * 3 * c) != cudaSuccess ||
                cudaMallocHost(&sv->h_off, sizeof(long long) * 3 * c) != cudaSuccess ||
                cudaMalloc(&sv->d_ins, sizeof(int) * c) != cudaSuccess ||
                cudaMallocHost(&sv->h_ins, sizeof(int) * c) != cudaSuccess)
                return VD_ERR_OOM;
            sv->off_cap = c;
        }
        // entry k spans [off[3k], off[3k + 3]) in each list; entry n holds the ends
        for (int k = 0; k < n; ++k) {
            const Retired& R = sv->retired[ts[k]];
            const bool ok = R.status == VD_OK && R.frame > 0;
            sv->h_ins[k] = sv->sims[R.sim].inst;
            sv->h_off[3 * k] = R.ob;
            sv->h_off[3 * k + 1] = R.oa;
            sv->h_off[3 * k + 2] = R.ok;
            sv->h_off[3 * k + 3] = R.ob + (ok ? R.nb : 0);
            sv->h_off[3 * k + 4] = R.oa + (ok ? R.na : 0);
            sv->h_off[3 * k + 5] = R.ok + (ok ? R.K : 0);
        }
        cudaError_t e = cudaMemcpyAsync(sv->d_off, sv->h_off, sizeof(long long) * 3 * (n + 1),
                                        cudaMemcpyHostToDevice, sv->cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sv->d_ins, sv->h_ins, sizeof(int) * n, cudaMemcpyHostToDevice, sv->cs);
        if (e != cudaSuccess) return VD_ERR_CUDA;
        r = vd_batch_gather_changes_list_async(sv->groups[gi].b, sv->cs, sv->d_ins, sv->d_off, n, nb,
                                               reinterpret_cast<uint64_t*>(sv->d_chg),
                                               sv->d_act);
        if (r) return r;
        // the host offset and instance buffers are reused by the next group
        if (cudaStreamSynchronize(sv->cs) != cudaSuccess) return VD_ERR_CUDA;
    }
    cudaError_t e = cudaSuccess;
    if (2 * nb + na > 0)
        e = cudaMemcpyAsync(sv->h_chg, sv->d_chg, sizeof(unsigned long long) * (2 * nb + na), cudaMemcpyDeviceToHost,
                            sv->cs);
    if (e == cudaSuccess && nk > 0) e = cudaMemcpyAsync(sv->h_act, sv->d_act, nk, cudaMemcpyDeviceToHost, sv->cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->cs);
    return e == cudaSuccess ? VD_OK : VD_ERR_CUDA;
}

vd_status copy_list(void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return VD_OK;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, dst) != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess ? VD_OK : VD_ERR_CUDA;
    std::memcpy(dst, src, bytes);
    return VD_OK;
}

}  // namespace

extern "C" {

vd_status vd_server_create(const vd_config* sims, int32_t n_sims, int64_t hbm_budget_bytes, int32_t max_batch,
                           void* stream, vd_server** out) {
    if (!out || n_sims < 0 || (n_sims > 0 && !sims) || hbm_budget_bytes <= 0 || max_batch < 1) return VD_ERR_INVALID;
    vd_server* sv = new (std::nothrow) vd_server();
    if (!sv) return VD_ERR_OOM;
    sv->max_batch = max_batch;
    sv->budget = hbm_budget_bytes;
    sv->s = (cudaStream_t)stream;
    if (n_sims > 0) {
        vd_status r = open_group(sv, sims, n_sims, nullptr);
        if (r) {
            delete sv;
            return r;
        }
    }
    *out = sv;
    return VD_OK;
}

vd_status vd_server_open_sim(vd_server* sv, const vd_config* cfg, int32_t* sim) {
    if (!sv || !cfg || !sim) return VD_ERR_INVALID;
    return open_group(sv, cfg, 1, sim);
}

vd_status vd_server_close_sim(vd_server* sv, int32_t sim) {
    if (!valid_sim(sv, sim)) return VD_ERR_INVALID;
    Sim& s = sv->sims[sim];
    if (s.busy || !s.q.empty()) return VD_ERR_STATE;
    s.open = false;
    Group& g = sv->groups[s.group];
    if (--g.open == 0) {
        // no instance of the group has work in flight; its memory leaves the budget
        vd_batch_destroy(g.b);
        g.b = nullptr;
        g.bytes = 0;
    }
    return VD_OK;
}

vd_status vd_server_clock_ns(int64_t* t) {
    if (!t) return VD_ERR_INVALID;
    *t = now_ns();
    return VD_OK;
}

vd_status vd_server_submit(vd_server* sv, int32_t sim, const float* d_field, int64_t t_arrival_ns, int64_t* ticket) {
    if (!valid_sim(sv, sim) || !d_field) return VD_ERR_INVALID;
    Pending p;
    p.ticket = sv->next_ticket++;
    p.field = d_field;
    p.t_submit = now_ns();
    p.t_arrival = t_arrival_ns > 0 ? t_arrival_ns : p.t_submit;
    p.bytes = 4ll * sv->sims[sim].cfg.Lx * sv->sims[sim].cfg.Ly;
    sv->sims[sim].q.push_back(p);
    if (ticket) *ticket = p.ticket;
    return VD_OK;
}

vd_status vd_server_keep_changes(vd_server* sv, int32_t on) {
    if (!sv) return VD_ERR_INVALID;
    if (on && !sv->cs && cudaStreamCreateWithFlags(&sv->cs, cudaStreamNonBlocking) != cudaSuccess) return VD_ERR_CUDA;
    sv->keep = on != 0;
    return VD_OK;
}

vd_status vd_server_poll(vd_server* sv, int32_t wait, vd_server_done* done, int32_t cap, int32_t* n_done) {
    if (!sv || (cap > 0 && !done)) return VD_ERR_INVALID;
    int nd = 0;
    vd_status r = VD_OK;
    sv->retired.clear();
    std::vector<long long> kept;
    for (;;) {
        // retire finished steps in launch order
        while (!sv->flight.empty()) {
            Step& st = sv->flight.front();
            const cudaError_t q = cudaEventQuery(st.done);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) return VD_ERR_CUDA;
            if (nd + (int)st.sims.size() > cap) break;   // caller's buffer is full: retire later
            const long long t = now_ns();
            const int* c = sv->h_cnt[st.slot];
            for (size_t k = 0; k < st.sims.size(); ++k) {
                vd_server_done& d = done[nd++];
                d.ticket = st.frames[k].ticket;
                d.sim = st.sims[k];
                d.t_arrival_ns = st.frames[k].t_arrival;
                d.t_submit_ns = st.frames[k].t_submit;
                d.t_done_ns = t;
                const int* ck = c + CNT * k;
                d.n_bubbles = ck[0];
                d.n_edges = ck[1];
                d.n_breaking = ck[2];
                d.n_arising = ck[3];
                d.status = ck[5] ? ((ck[5] & 16) ? VD_ERR_TIMEOUT : VD_ERR_CAPACITY) : VD_OK;
                sv->sims[st.sims[k]].busy = false;
                sv->inflight_bytes -= st.frames[k].bytes;
                if (sv->keep) {
                    Retired R;
                    std::memset(&R, 0, sizeof(R));
                    R.sim = st.sims[k];
                    R.status = d.status;
                    R.K = d.n_bubbles;
                    R.n_edges = d.n_edges;
                    R.nb = d.n_breaking;
                    R.na = d.n_arising;
                    R.n_matched = ck[4];
                    R.n_prev = ck[6];
                    R.frame = ck[7];
                    sv->retired[d.ticket] = R;
                    kept.push_back(d.ticket);
                }
            }
            sv->slot_busy[st.slot] = 0;
            sv->frames_done += (long long)st.sims.size();
            sv->ev_free.push_back(st.done);
            sv->flight.pop_front();
        }
        if (sv->keep && !kept.empty()) {
            r = keep_retired(sv, kept);
            if (r) break;
            kept.clear();
        }
        // keep up to two steps queued on the device
        while (sv->flight.size() < 2) {
            const size_t before = sv->flight.size();
            r = server_launch(sv);
            if (r || sv->flight.size() == before) break;
        }
        if (r) break;
        if (!wait || nd > 0 || sv->flight.empty()) break;
    }
    if (n_done) *n_done = nd;
    return r;
}

vd_status vd_server_get_frame_changes(vd_server* sv, int64_t ticket, vd_changes* out) {
    if (!sv || !out) return VD_ERR_INVALID;
    auto it = sv->retired.find(ticket);
    if (it == sv->retired.end()) return VD_ERR_STATE;
    const Retired& R = it->second;
    out->frame_index = R.frame - 1;
    out->n_prev = R.n_prev;
    out->n_now = R.K;
    out->n_matched = R.n_matched;
    out->n_edges = R.n_edges;
    out->n_breaking = R.nb;
    out->n_arising = R.na;
    out->global_trigger = (R.nb + R.na) > 0;
    if (R.status) return R.status;
    if (R.frame <= 0) return VD_ERR_STATE;
    if ((R.nb > 0 && (!out->breaking || out->cap_breaking < R.nb)) ||
        (R.na > 0 && (!out->arising || out->cap_arising < R.na)) || (out->active && out->cap_active < R.K))
        return VD_ERR_CAPACITY;
    const size_t u8 = sizeof(unsigned long long);
    vd_status r = VD_OK;
    if (R.nb > 0) {
        r = copy_list(out->breaking, sv->h_chg + R.ob, u8 * R.nb);
        if (!r && out->breaking_prev) r = copy_list(out->breaking_prev, sv->h_chg + sv->chg_nb + R.ob, u8 * R.nb);
    }
    if (!r && R.na > 0) r = copy_list(out->arising, sv->h_chg + 2 * sv->chg_nb + R.oa, u8 * R.na);
    if (!r && out->active && R.K > 0) r = copy_list(out->active, sv->h_act + R.ok, R.K);
    return r;
}

vd_status vd_server_get_changes(vd_server* sv, int32_t sim, vd_changes* out) {
    if (!valid_sim(sv, sim)) return VD_ERR_INVALID;
    const Sim& s = sv->sims[sim];
    if (s.busy) return VD_ERR_STATE;   // a frame of this simulation is still in flight
    return vd_batch_get_changes(sv->groups[s.group].b, s.inst, out);
}

vd_status vd_server_get_labels(vd_server* sv, int32_t sim, int32_t* out, int64_t cap, int64_t* n) {
    if (!valid_sim(sv, sim)) return VD_ERR_INVALID;
    const Sim& s = sv->sims[sim];
    if (s.busy) return VD_ERR_STATE;
    return vd_batch_get_labels(sv->groups[s.group].b, s.inst, out, cap, n);
}

vd_status vd_server_export_state(vd_server* sv, int32_t sim, void* buf, int64_t cap, int64_t* n_bytes) {
    if (!valid_sim(sv, sim)) return VD_ERR_INVALID;
    const Sim& s = sv->sims[sim];
    if (s.busy) return VD_ERR_STATE;
    return vd_batch_export_state(sv->groups[s.group].b, s.inst, buf, cap, n_bytes);
}

vd_status vd_server_import_state(vd_server* sv, int32_t sim, const void* buf, int64_t n_bytes) {
    if (!valid_sim(sv, sim)) return VD_ERR_INVALID;
    const Sim& s = sv->sims[sim];
    if (s.busy || !s.q.empty()) return VD_ERR_STATE;
    return vd_batch_import_state(sv->groups[s.group].b, s.inst, buf, n_bytes);
}

vd_status vd_server_stats(vd_server* sv, int64_t* steps, int64_t* frames_done, int64_t* resident_bytes,
                          int64_t* queued) {
    if (!sv) return VD_ERR_INVALID;
    if (steps) *steps = sv->steps;
    if (frames_done) *frames_done = sv->frames_done;
    if (resident_bytes) *resident_bytes = resident(sv);
    if (queued) {
        long long qn = 0;
        for (const Sim& s : sv->sims) qn += (long long)s.q.size();
        *queued = qn;
    }
    return VD_OK;
}

vd_status vd_server_destroy(vd_server* sv) {
    if (!sv) return VD_ERR_INVALID;
    cudaStreamSynchronize(sv->s);
    for (auto& st : sv->flight) cudaEventDestroy(st.done);
    for (cudaEvent_t e : sv->ev_free) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        cudaFree(sv->d_cnt[k]);
        cudaFreeHost(sv->h_cnt[k]);
    }
    if (sv->cs) {
        cudaStreamSynchronize(sv->cs);
        cudaStreamDestroy(sv->cs);
    }
    cudaFree(sv->d_chg);
    cudaFreeHost(sv->h_chg);
    cudaFree(sv->d_act);
    cudaFreeHost(sv->h_act);
    cudaFree(sv->d_off);
    cudaFreeHost(sv->h_off);
    cudaFree(sv->d_ins);
    cudaFreeHost(sv->h_ins);
    for (Group& g : sv->groups)
        if (g.b) vd_batch_destroy(g.b);
    delete sv;
    return VD_OK;
}

}  // extern "C"
