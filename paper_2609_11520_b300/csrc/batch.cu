// Batched online stage over several resident operators of uneven size:
// F_i = G~_i^{-1} K~_i^* U_i for operators i = 0..n-1 (Eq. 4.2 for each).
//
// Execution modes:
//   0  one fio_solve per operator (about 20 launches each);
//   1  grouped launches: one launch per stage covers every operator -- the
//      two fused BF half passes, one ULV node-product launch per tree depth
//      (up pass by distance from the leaves, down pass by level), and one
//      launch for all roots -- driven by device tables of per-operator
//      arguments and flattened work items built once per plan;
//   2  mode 1 captured into a CUDA graph on the first solve of a plan and
//      replayed afterwards.
// A plan is keyed by the U / F pointers and column counts; a new key replans.
// fio_batch_autotune times the candidate configurations on the caller's
// buffers (per-operator kernel path for mode 0: fused staged, fused
// unstaged, one kernel per factor; modes 1 and 2) and keeps the fastest.
#include <algorithm>
#include <cstring>

#include "bf.cuh"
#include "hss.cuh"

struct fio_batch {
    std::vector<fio_bf*> bfs;
    std::vector<fio_hss*> hss;
    int mode = 2;
    int path0 = 0;   // bf_set_path value used by mode 0
    // current plan
    bool planned = false;
    std::vector<const void*> keyU;
    std::vector<void*> keyF;
    std::vector<int> keyK;
    fio::DevBuf T, mid, ulvws;                // K~^* U, BF middle states, ULV solve vectors (per operator)
    std::vector<int> fallback;                // operators not covered by the grouped BF kernels
    int bfmode = 0;                           // transfer-level mode of the grouped BF kernels (bf_fused_mode)
    std::vector<size_t> Toff;
    fio::DevBuf dargs_l, dargs_r, ditems_l, ditems_r;
    int nl = 0, nr = 0;
    fio::DevBuf ddesc, ditems, droots;
    std::vector<int> up_off, up_cnt, dn_off, dn_cnt;   // item ranges per launch
    int nroots = 0;
    // persistent mode: work list and its counters
    fio::DevBuf ditems_p, dctr_p;
    int nitems_p = 0, nctr_p = 0;
    int spin_limit = 1 << 20;   // polls of a dependency wait (~0.1 s at the poll interval)
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t capture_stream = nullptr;   // private: the caller's stream may be the legacy default stream
};

namespace fio {
namespace {

template <class T> fio_status upload(DevBuf& b, const std::vector<T>& v) {
    FIO_TRY(b.ensure(std::max<size_t>(16, v.size() * sizeof(T))));
    if (!v.empty()) FIO_CUDA(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FIO_OK;
}

void drop_graph(fio_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
}

fio_status plan(fio_batch* b, const void* const* U, void* const* F, const int* k) {
    const int n = int(b->bfs.size());
    drop_graph(b);
    b->planned = false;
    b->keyU.assign(U, U + n);
    b->keyF.assign(F, F + n);
    b->keyK.assign(k, k + n);
    // per-operator buffers
    size_t tT = 0, tM = 0;
    std::vector<size_t> moff(n);
    b->Toff.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        b->Toff[i] = tT;
        moff[i] = tM;
        tT += size_t(b->bfs[i]->n) * k[i];
        tM += size_t(b->bfs[i]->n) * b->bfs[i]->r * k[i];
    }
    FIO_TRY(b->T.ensure(std::max<size_t>(16, tT * 8)));
    FIO_TRY(b->mid.ensure(std::max<size_t>(16, tM * 8)));
    // grouped BF adjoint
    std::vector<BfGroupOp> ops;
    b->fallback.clear();
    b->bfmode = -1;   // the grouped launch runs one transfer-level mode: the first covered operator's
    for (int i = 0; i < n; ++i) {
        if (k[i] == 0) continue;
        if (bf_v3_ok(b->bfs[i]) && b->bfmode < 0) b->bfmode = bf_fused_mode(b->bfs[i], -1);
        if (bf_v3_ok(b->bfs[i]) && bf_fused_mode(b->bfs[i], -1) == b->bfmode)
            ops.push_back(BfGroupOp{b->bfs[i], static_cast<const float2*>(U[i]), b->T.as<float2>() + b->Toff[i],
                                    b->mid.as<float2>() + moff[i], k[i]});
        else
            b->fallback.push_back(i);
    }
    if (b->bfmode < 0) b->bfmode = 0;
    std::vector<unsigned char> la, ra;
    std::vector<int4> li, ri;
    bf_group_tables(ops, 1, la, li, ra, ri);
    FIO_TRY(upload(b->dargs_l, la));
    FIO_TRY(upload(b->dargs_r, ra));
    FIO_TRY(upload(b->ditems_l, li));
    FIO_TRY(upload(b->ditems_r, ri));
    b->nl = int(li.size());
    b->nr = int(ri.size());
    // grouped ULV solve
    std::vector<UlvSolvePlan> plans(n);
    std::vector<int64_t> woff(n, 0);
    int64_t wtot = 0;
    for (int i = 0; i < n; ++i) {
        woff[i] = wtot;
        if (k[i] > 0) wtot += ulv_solve_ws_elems(b->hss[i], k[i]);
    }
    FIO_TRY(b->ulvws.ensure(std::max<size_t>(16, size_t(wtot) * 8)));
    int maxLh = 0;
    for (int i = 0; i < n; ++i) {
        if (k[i] == 0) continue;
        FIO_TRY(ulv_solve_plan(b->hss[i], b->T.as<float2>() + b->Toff[i], static_cast<float2*>(F[i]), b->bfs[i]->n, k[i],
                               b->ulvws.as<float2>() + woff[i], plans[i]));
        maxLh = std::max(maxLh, plans[i].Lh);
    }
    std::vector<UlvGemmDesc> descs;
    std::vector<int4> items;
    std::vector<UlvRootDesc> roots;
    b->up_off.assign(maxLh, 0);
    b->up_cnt.assign(maxLh, 0);
    b->dn_off.assign(maxLh + 1, 0);
    b->dn_cnt.assign(maxLh + 1, 0);
    for (int d = 0; d < maxLh; ++d) {   // up pass: distance d from the leaves
        b->up_off[d] = int(items.size());
        for (int i = 0; i < n; ++i) {
            if (k[i] == 0 || plans[i].Lh <= d) continue;
            const UlvGemmDesc& g = plans[i].up[plans[i].Lh - d];
            if (g.nodes == 0) continue;
            descs.push_back(g);
            ulv_gemm_items(g, int(descs.size()) - 1, items);
        }
        b->up_cnt[d] = int(items.size()) - b->up_off[d];
    }
    for (int i = 0; i < n; ++i)
        if (k[i] > 0 && plans[i].root.m > 0) roots.push_back(plans[i].root);
    for (int l = 1; l <= maxLh; ++l) {   // down pass: level l
        b->dn_off[l] = int(items.size());
        for (int i = 0; i < n; ++i) {
            if (k[i] == 0 || plans[i].Lh < l) continue;
            const UlvGemmDesc& g = plans[i].down[l];
            if (g.nodes == 0) continue;
            descs.push_back(g);
            ulv_gemm_items(g, int(descs.size()) - 1, items);
        }
        b->dn_cnt[l] = int(items.size()) - b->dn_off[l];
    }
    // ---- persistent work list: stages in dependency order, each item waiting on the counter of
    // the previous stage of its own operator
    {
        std::vector<PItem> pl;
        int nctr = 0;
        std::vector<int> last_ctr(n, -1), last_target(n, 0);
        std::vector<int> bidx;   // batch index of each grouped BF operator
        for (int i = 0; i < n; ++i)
            if (k[i] > 0 && std::find(b->fallback.begin(), b->fallback.end(), i) == b->fallback.end()) bidx.push_back(i);
        const int nops = int(bidx.size());
        std::vector<int> cl(nops, -1), nl(nops, 0), cr(nops, -1), nr(nops, 0);
        for (const int4& v : li) {
            if (cl[v.x] < 0) cl[v.x] = nctr++;
            pl.push_back(PItem{kPLeft, v.x, v.y, v.z, 0, -1, 0, 0, -1, 0, cl[v.x], 0});
            ++nl[v.x];
        }
        for (const int4& v : ri) {
            if (cr[v.x] < 0) cr[v.x] = nctr++;
            pl.push_back(PItem{kPRight, v.x, v.y, v.z, 0, -1, 0, 0, cl[v.x], nl[v.x], cr[v.x], 0});
            ++nr[v.x];
        }
        for (int o = 0; o < nops; ++o) {
            last_ctr[bidx[o]] = cr[o];
            last_target[bidx[o]] = nr[o];
        }
        // node-product blocks of a stage go two to an item (one per half of the CTA)
        auto add_stage = [&](int i, int type, const std::vector<int4>& its) {
            if (its.empty()) return;
            const int c = nctr++;
            int cnt = 0;
            const bool pair = type == kPUp || type == kPDown;
            for (size_t j = 0; j < its.size(); j += pair ? 2 : 1) {
                const int4 v = its[j];
                PItem it{type, v.x, v.y, v.z, v.w, -1, 0, 0, last_ctr[i], last_target[i], c, 0};
                if (pair && j + 1 < its.size()) {
                    it.b2 = its[j + 1].y;
                    it.c2 = its[j + 1].z;
                    it.d2 = its[j + 1].w;
                }
                pl.push_back(it);
                ++cnt;
            }
            last_ctr[i] = c;
            last_target[i] = cnt;
        };
        std::vector<UlvGemmDesc> pdesc;
        std::vector<UlvRootDesc> proots;
        for (int d = 0; d < maxLh; ++d)
            for (int i = 0; i < n; ++i) {
                if (k[i] == 0 || plans[i].Lh <= d) continue;
                const UlvGemmDesc& g = plans[i].up[plans[i].Lh - d];
                if (g.nodes == 0) continue;
                pdesc.push_back(g);
                std::vector<int4> its;
                ulv_gemm_items(g, int(pdesc.size()) - 1, its);
                add_stage(i, kPUp, its);
            }
        for (int i = 0; i < n; ++i)
            if (k[i] > 0 && plans[i].root.m > 0) {
                proots.push_back(plans[i].root);
                add_stage(i, kPRoot, {make_int4(int(proots.size()) - 1, 0, 0, 0)});
            }
        for (int l = 1; l <= maxLh; ++l)
            for (int i = 0; i < n; ++i) {
                if (k[i] == 0 || plans[i].Lh < l) continue;
                const UlvGemmDesc& g = plans[i].down[l];
                if (g.nodes == 0) continue;
                pdesc.push_back(g);
                std::vector<int4> its;
                ulv_gemm_items(g, int(pdesc.size()) - 1, its);
                add_stage(i, kPDown, its);
            }
        // the persistent list's own descriptor arrays follow the grouped ones in device memory
        const int d0 = int(descs.size()), r0 = int(roots.size());
        for (PItem& it : pl) {
            if (it.type == kPUp || it.type == kPDown) it.a += d0;
            if (it.type == kPRoot) it.a += r0;
        }
        b->nroots = r0;
        descs.insert(descs.end(), pdesc.begin(), pdesc.end());
        roots.insert(roots.end(), proots.begin(), proots.end());
        FIO_TRY(upload(b->ditems_p, pl));
        FIO_TRY(b->dctr_p.ensure(size_t(1 + nctr) * sizeof(int)));
        b->nitems_p = int(pl.size());
        b->nctr_p = nctr;
    }
    FIO_TRY(upload(b->ddesc, descs));
    FIO_TRY(upload(b->ditems, items));
    FIO_TRY(upload(b->droots, roots));
    b->planned = true;
    return FIO_OK;
}

fio_status launch_grouped(fio_batch* b, cudaStream_t st) {
    FIO_TRY(bf_group_launch(b->dargs_l.p, b->ditems_l.as<int4>(), b->nl, b->dargs_r.p, b->ditems_r.as<int4>(), b->nr, 1,
                            b->bfmode, st));
    for (int i : b->fallback)
        FIO_TRY(bf_apply(b->bfs[i], b->keyU[i], b->T.as<float2>() + b->Toff[i], b->bfs[i]->n, b->keyK[i], 1, st));
    const int4* it = b->ditems.as<int4>();
    const UlvGemmDesc* dd = b->ddesc.as<UlvGemmDesc>();
    for (size_t d = 0; d < b->up_off.size(); ++d)
        FIO_TRY(ulv_group_launch(dd, it + b->up_off[d], b->up_cnt[d], false, st));
    FIO_TRY(ulv_root_group_launch(b->droots.as<UlvRootDesc>(), b->nroots, st));
    for (size_t l = 1; l < b->dn_off.size(); ++l)
        FIO_TRY(ulv_group_launch(dd, it + b->dn_off[l], b->dn_cnt[l], true, st));
    return FIO_OK;
}

// One persistent launch over the whole work list (after the K~^* of any operator the grouped
// BF kernels do not cover).
fio_status launch_persistent(fio_batch* b, cudaStream_t st) {
    for (int i : b->fallback)
        FIO_TRY(bf_apply(b->bfs[i], b->keyU[i], b->T.as<float2>() + b->Toff[i], b->bfs[i]->n, b->keyK[i], 1, st));
    return batch_persistent_launch(b->dargs_l.p, b->dargs_r.p, b->ddesc.as<UlvGemmDesc>(), b->droots.as<UlvRootDesc>(),
                                   b->ditems_p.as<PItem>(), b->nitems_p, b->dctr_p.as<int>(), b->nctr_p, b->bfmode,
                                   b->spin_limit, st);
}

bool same_key(const fio_batch* b, const void* const* U, void* const* F, const int* k) {
    const size_t n = b->bfs.size();
    for (size_t i = 0; i < n; ++i)
        if (b->keyU[i] != U[i] || b->keyF[i] != F[i] || b->keyK[i] != k[i]) return false;
    return true;
}

}  // namespace
}  // namespace fio

using namespace fio;

extern "C" fio_status fio_batch_create(fio_bf* const* bfs, fio_hss* const* hss, int n_ops, fio_batch** out) {
    if (!out || !bfs || !hss || n_ops < 1) return fail(FIO_EINVAL, "fio_batch_create: bad arguments");
    *out = nullptr;
    for (int i = 0; i < n_ops; ++i) {
        if (!bfs[i] || !hss[i]) return fail(FIO_EINVAL, "fio_batch_create: null operator");
        if (bfs[i]->N() != hss[i]->N) return fail(FIO_EINVAL, "fio_batch_create: BF and HSS sizes differ");
        if (!hss[i]->factored) return fail(FIO_EINVAL, "fio_batch_create: HSS not factored");
        if (bfs[i]->d != 1) return fail(FIO_EINVAL, "fio_batch_create: 1D operators only (2D: fio_solve)");
    }
    fio_batch* b = new fio_batch();
    b->bfs.assign(bfs, bfs + n_ops);
    b->hss.assign(hss, hss + n_ops);
    *out = b;
    return FIO_OK;
}

extern "C" fio_status fio_batch_set_mode(fio_batch* b, int mode) {
    if (!b || mode < 0 || mode > 3) return fail(FIO_EINVAL, "fio_batch_set_mode: bad mode");
    b->mode = mode;
    return FIO_OK;
}

extern "C" fio_status fio_batch_solve(fio_batch* b, const void* const* U, void* const* F, const int* k, void* stream) {
    if (!b || !U || !F || !k) return fail(FIO_EINVAL, "fio_batch_solve: null argument");
    const int n = int(b->bfs.size());
    for (int i = 0; i < n; ++i) {
        if (k[i] < 0) return fail(FIO_EINVAL, "fio_batch_solve: negative k");
        if (k[i] > 0 && (!U[i] || !F[i])) return fail(FIO_EINVAL, "fio_batch_solve: null vector");
    }
    cudaStream_t st = as_stream(stream);
    if (b->mode == 0) {
        for (int i = 0; i < n; ++i) {
            if (k[i] == 0) continue;
            FIO_TRY(bf_set_path(b->bfs[i], b->path0));
            FIO_TRY(fio_solve(b->bfs[i], b->hss[i], U[i], F[i], b->bfs[i]->n, k[i], 0, st));
        }
        return FIO_OK;
    }
    if (!b->planned || !same_key(b, U, F, k)) FIO_TRY(plan(b, U, F, k));
    if (b->mode == 1) return launch_grouped(b, st);
    if (b->mode == 3) return launch_persistent(b, st);
    if (!b->gexec) {
        FIO_TRY(launch_grouped(b, st));   // first run eagerly (also sets kernel attributes)
        FIO_CUDA(cudaStreamSynchronize(st));
        if (!b->capture_stream) FIO_CUDA(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
        cudaStream_t cs = b->capture_stream;
        FIO_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        fio_status s = launch_grouped(b, cs);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (s != FIO_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return cuda_status(e, "fio_batch_solve: stream capture");
        b->graph = g;
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        if (e != cudaSuccess) {
            drop_graph(b);
            return cuda_status(e, "fio_batch_solve: graph instantiation");
        }
        return FIO_OK;   // this call's results came from the eager run
    }
    FIO_CUDA(cudaGraphLaunch(b->gexec, st));
    return FIO_OK;
}

extern "C" fio_status fio_batch_autotune(fio_batch* b, const void* const* U, void* const* F, const int* k, int reps,
                                         void* stream, char* report, int64_t len) {
    if (!b || reps < 1) return fail(FIO_EINVAL, "fio_batch_autotune: bad arguments");
    cudaStream_t st = as_stream(stream);
    // knobs: launch structure (per operator / grouped / graph / one persistent launch), BF kernels
    // of the per-operator mode, and the transfer-level arithmetic (tensor cores or CUDA cores)
    struct Cand {
        int mode, path, simt;
        const char* name;
    };
    const Cand cands[] = {{0, 2, 0, "per-operator, fused staged"},
                          {0, 3, 0, "per-operator, fused unstaged"},
                          {0, 1, 0, "per-operator, one kernel per factor"},
                          {1, 0, 0, "grouped launches"},
                          {2, 0, 0, "grouped launches in a CUDA graph"},
                          {3, 0, 0, "one persistent launch over a work list"},
                          {1, 0, 1, "grouped launches, CUDA-core transfer levels"},
                          {3, 0, 1, "one persistent launch, CUDA-core transfer levels"}};
    std::vector<bool> simt0;
    for (auto* bf : b->bfs) simt0.push_back(bf->simt);
    auto set_simt = [&](int v) {
        for (auto* bf : b->bfs)
            if (bf_v3_ok(bf)) bf->simt = v != 0;
        b->planned = false;
        drop_graph(b);
    };
    cudaEvent_t e0, e1;
    FIO_CUDA(cudaEventCreate(&e0));
    FIO_CUDA(cudaEventCreate(&e1));
    std::string rep;
    float best = 1e30f;
    int bi = -1;
    for (int c = 0; c < int(sizeof(cands) / sizeof(cands[0])); ++c) {
        b->mode = cands[c].mode;
        b->path0 = cands[c].path;
        set_simt(cands[c].simt);
        bool ok = true;
        if (cands[c].mode == 0)
            for (auto* bf : b->bfs)
                if (cands[c].path >= 2 && !bf_fused_ok(bf)) ok = false;
        if (!ok) continue;
        fio_status s = fio_batch_solve(b, U, F, k, st);   // warm (plans, captures)
        if (s == FIO_OK) s = fio_batch_solve(b, U, F, k, st);
        if (s != FIO_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return s;
        }
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) fio_batch_solve(b, U, F, k, st);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_status(e, "fio_batch_autotune");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        rep += std::string(cands[c].name) + " " + std::to_string(ms) + " ms\n";
        if (ms < best) {
            best = ms;
            bi = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bi < 0) return fail(FIO_EINVAL, "fio_batch_autotune: no candidate applies");
    b->mode = cands[bi].mode;
    b->path0 = cands[bi].path;
    for (size_t i = 0; i < b->bfs.size(); ++i) {
        bf_set_path(b->bfs[i], 0);
        b->bfs[i]->simt = simt0[i];
    }
    if (cands[bi].simt) set_simt(1);
    b->planned = false;
    drop_graph(b);
    rep += std::string("chosen: ") + cands[bi].name + "\n";
    if (report && len > 0) {
        std::strncpy(report, rep.c_str(), size_t(len) - 1);
        report[len - 1] = 0;
    }
    return FIO_OK;
}

extern "C" void fio_batch_free(fio_batch* b) {
    if (!b) return;
    drop_graph(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (DevBuf* d : {&b->T, &b->mid, &b->ulvws, &b->dargs_l, &b->dargs_r, &b->ditems_l, &b->ditems_r, &b->ddesc, &b->ditems,
                      &b->droots})
        d->release();
    delete b;
}

extern "C" fio_status fio_selftest_wait_timeout(void* stream) {
    // A one-item work list whose prerequisite counter nothing increments: the item's bounded wait
    // must run out (about 1000 polls), set the device flag and let the kernel finish.
    cudaStream_t st = as_stream(stream);
    fio::DevBuf d_items, d_root, d_ctr;
    auto release = [&]() {
        d_items.release();
        d_root.release();
        d_ctr.release();
    };
    const PItem it{kPRoot, 0, 0, 0, 0, -1, 0, 0, 0, 1, 1, 0};
    const UlvRootDesc rd{nullptr, nullptr, nullptr, 0, 0};
    fio_status s = upload(d_items, std::vector<PItem>{it});
    if (s == FIO_OK) s = upload(d_root, std::vector<UlvRootDesc>{rd});
    if (s == FIO_OK) s = d_ctr.ensure(3 * sizeof(int));
    if (s == FIO_OK)
        s = batch_persistent_launch(nullptr, nullptr, nullptr, d_root.as<UlvRootDesc>(), d_items.as<PItem>(), 1,
                                    d_ctr.as<int>(), 2, 1, 1000, st);
    if (s == FIO_OK) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_status(e, "fio_selftest_wait_timeout");
    }
    release();
    if (s != FIO_OK) return s;
    return fio_device_status();
}
