// batch.cu -- many independent cases in one CUDA graph, and the autotuner of
// the launch shapes.
//
// A batch captures two pdf_steps of every context into a single graph: a fork
// event on the batch stream, every context's steps on its own stream, a join
// back. Replaying the graph launches all cases' kernels with one call; cases
// of uneven size overlap on the GPU. Two steps, because the re-sort moves the
// particle state between two buffers and swaps them on the host: a captured
// pair of steps starts and ends in the same buffers. The step counter of every context lives
// on the device (advanced by the re-sort), so replays draw new Philox streams.
// Cooperative CG grids are chained with an event (one resident at a time):
// two partially resident cooperative grids waiting at their grid barriers
// could otherwise starve each other. The capture goes step by step over the
// contexts (every context's first step, then every context's second), so the
// chain runs through all first-step solves before any second-step one and a
// context never waits for another context's later step.
#include <algorithm>
#include <vector>

#include "pdf_internal.cuh"

struct pdf_batch {
    std::vector<pdf_ctx*> ctx;
    cudaStream_t s = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;
    std::vector<int64_t> launches;  // kernels of one captured step, per context
};

namespace {

void release(pdf_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    delete b;
}

int cuda_fail(const char* what, cudaError_t e) {
    return fail(nullptr, PDF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

// the field mapping of pdf_get_fields (api.cu)
int field_source(pdf_ctx* c, int32_t field, const void** src, size_t* need, bool* convert);

extern "C" {

int pdf_batch_create_out(pdf_ctx* const* ctx, const double* dt, int32_t n, void* cuda_stream, int32_t field,
                         void* const* fout, const size_t* fbytes, pdf_batch** out) {
    if (!out) return fail(nullptr, PDF_ERR_ARG, "pdf_batch_create: out is NULL");
    *out = nullptr;
    if (!ctx || !dt || n < 1 || !cuda_stream) return fail(nullptr, PDF_ERR_ARG, "pdf_batch_create: bad arguments");
    if (fout && !fbytes) return fail(nullptr, PDF_ERR_ARG, "pdf_batch_create_out: bytes is NULL");
    for (int i = 0; fout && i < 2 * n; ++i)
        if (!fout[i]) return fail(nullptr, PDF_ERR_ARG, "pdf_batch_create_out: NULL output buffer");
    for (int i = 0; i < n; ++i) {
        pdf_ctx* c = ctx[i];
        if (!c || !c->s || c->s == (cudaStream_t)cuda_stream || !(dt[i] > 0) || !c->stats_valid)
            return fail(nullptr, PDF_ERR_ARG, "pdf_batch_create: context " + std::to_string(i) +
                                                  " needs its own stream, a positive dt and estimated statistics");
        for (int j = 0; j < i; ++j)
            if (ctx[j] == c || ctx[j]->s == c->s)
                return fail(nullptr, PDF_ERR_ARG, "pdf_batch_create: contexts and streams must be distinct");
    }
    // output sizes checked before the capture (a failure inside it would leave
    // a context with a step captured and its state buffers swapped)
    for (int i = 0; fout && i < n; ++i) {
        const void* src = nullptr;
        size_t need = 0;
        bool convert = false;
        const int st = field_source(ctx[i], field, &src, &need, &convert);
        if (st != PDF_OK) return fail(nullptr, st, "pdf_batch_create_out: context " + std::to_string(i) + ": " + ctx[i]->err);
        if (fbytes[i] != need)
            return fail(nullptr, PDF_ERR_ARG, "pdf_batch_create_out: context " + std::to_string(i) +
                                                  ": field size mismatch, expected " + std::to_string(need));
    }
    // launch set-up outside the capture
    for (int i = 0; i < n; ++i) {
        pdf_ctx* c = ctx[i];
        int st = c->step_blocks ? PDF_OK : prepare_particle(c, 0);
        if (st == PDF_OK && c->p.wall_model == PDF_ELLIPTIC_RELAXATION && !c->fe_blocks) st = prepare_elliptic(c, 0);
        if (st != PDF_OK) return fail(nullptr, st, "pdf_batch_create: context " + std::to_string(i) + ": " + c->err);
    }
    pdf_batch* b = new pdf_batch;
    b->ctx.assign(ctx, ctx + n);
    b->s = (cudaStream_t)cuda_stream;
    b->ev.resize(1 + 2 * (size_t)n);
    b->launches.assign(n, 0);
    for (auto& e : b->ev) {
        const cudaError_t err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (err != cudaSuccess) {
            e = nullptr;
            release(b);
            return cuda_fail("cudaEventCreateWithFlags", err);
        }
    }
    cudaEvent_t fork = b->ev[0], chain = b->ev[1 + n];
    cudaError_t err = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeRelaxed);
    if (err != cudaSuccess) {
        release(b);
        return cuda_fail("cudaStreamBeginCapture", err);
    }
    // the host-side step state of every context (a captured step advances the
    // step counter and swaps the state buffers as if it had run): restored
    // below if the capture fails part of the way
    struct Saved {
        int step;
        void *a[7], *b[7];
        uint32_t *ia, *ib;
        int *ea, *eb;
    };
    std::vector<Saved> saved((size_t)n);
    for (int i = 0; i < n; ++i) {
        Saved& v = saved[(size_t)i];
        v.step = ctx[i]->step;
        for (int q = 0; q < 7; ++q) { v.a[q] = ctx[i]->stA[q]; v.b[q] = ctx[i]->stB[q]; }
        v.ia = ctx[i]->idA; v.ib = ctx[i]->idB; v.ea = ctx[i]->elemA; v.eb = ctx[i]->elemB;
    }
    auto restore = [&]() {
        for (int i = 0; i < n; ++i) {
            const Saved& v = saved[(size_t)i];
            ctx[i]->step = v.step;
            for (int q = 0; q < 7; ++q) { ctx[i]->stA[q] = v.a[q]; ctx[i]->stB[q] = v.b[q]; }
            ctx[i]->idA = v.ia; ctx[i]->idB = v.ib; ctx[i]->elemA = v.ea; ctx[i]->elemB = v.eb;
        }
    };
    int st = PDF_OK;
    err = cudaEventRecord(fork, b->s);
    for (int i = 0; i < n && err == cudaSuccess; ++i) err = cudaStreamWaitEvent(ctx[i]->s, fork, 0);
    bool chained = false;  // a cooperative solve has been captured (the chain event holds it)
    for (int k = 0; k < 2 && st == PDF_OK && err == cudaSuccess; ++k) {
        for (int i = 0; i < n && st == PDF_OK && err == cudaSuccess; ++i) {
            pdf_ctx* c = ctx[i];
            const int timing = c->timing;
            c->timing = 0;
            const int64_t l0 = c->launches;
            c->coop_wait = chained ? chain : nullptr;
            c->coop_done = chain;
            st = pdf_step(c, dt[i], 1);
            if (c->launches > l0 && (c->p.wall_model == PDF_ELLIPTIC_RELAXATION || c->p.pressure)) chained = true;
            // the requested field after this step: an asynchronous device copy on
            // the context stream, captured as a node of the graph
            if (st == PDF_OK && fout) st = pdf_get_fields(c, field, fout[2 * i + k], fbytes[i], 1);
            b->launches[i] += c->launches - l0;
            c->launches = l0;
            c->coop_wait = c->coop_done = nullptr;
            c->timing = timing;
            if (st == PDF_OK) c->step -= 1;  // captured, not executed
            else st = fail(nullptr, st, "pdf_batch_create: step of context " + std::to_string(i) + ": " + c->err);
        }
    }
    for (int i = 0; i < n && st == PDF_OK && err == cudaSuccess; ++i) {
        err = cudaEventRecord(b->ev[1 + i], ctx[i]->s);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(b->s, b->ev[1 + i], 0);
    }
    const cudaError_t end = cudaStreamEndCapture(b->s, &b->graph);
    if (st != PDF_OK || err != cudaSuccess || end != cudaSuccess) {
        restore();  // nothing of the capture ran: every context stays where it was
        release(b);
        if (st != PDF_OK) return st;
        return cuda_fail("stream capture of the batch step", err != cudaSuccess ? err : end);
    }
    err = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (err != cudaSuccess) {
        release(b);
        return cuda_fail("cudaGraphInstantiate", err);
    }
    *out = b;
    return PDF_OK;
}

int pdf_batch_step(pdf_batch* b, int32_t nsteps) {
    if (!b || nsteps < 0 || (nsteps & 1))
        return fail(nullptr, PDF_ERR_ARG, "pdf_batch_step: nsteps must be even and >= 0");
    for (int k = 0; k < nsteps / 2; ++k) {
        const cudaError_t err = cudaGraphLaunch(b->exec, b->s);
        if (err != cudaSuccess) return cuda_fail("cudaGraphLaunch", err);
    }
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        b->ctx[i]->step += nsteps;
        b->ctx[i]->launches += b->launches[i] * (nsteps / 2);
    }
    return PDF_OK;
}

int pdf_batch_sync(pdf_batch* b, int32_t* failed) {
    if (!b) return PDF_ERR_ARG;
    if (failed) *failed = -1;
    const cudaError_t err = cudaStreamSynchronize(b->s);
    if (err != cudaSuccess) return cuda_fail("cudaStreamSynchronize", err);
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        const int st = pdf_sync(b->ctx[i]);
        if (st != PDF_OK) {
            if (failed) *failed = (int32_t)i;
            return st;
        }
    }
    return PDF_OK;
}

int pdf_batch_create(pdf_ctx* const* ctx, const double* dt, int32_t n, void* cuda_stream, pdf_batch** out) {
    return pdf_batch_create_out(ctx, dt, n, cuda_stream, 0, nullptr, nullptr, out);
}

void pdf_batch_destroy(pdf_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->s);
    release(b);
}

int pdf_autotune(pdf_ctx* c, double dt, int32_t steps_per_trial, pdf_tuning* out) {
    if (!c || !(dt > 0) || steps_per_trial < 1) return PDF_ERR_ARG;
    if (!c->stats_valid) return fail(c, PDF_ERR_STATE, "statistics not estimated");
    const int timing = c->timing;
    c->timing = 1;
    auto trial = [&](int kernel, double& ms) -> int {
        int st = pdf_step(c, dt, 1);  // warm-up with the new shape
        if (st == PDF_OK) st = pdf_reset_timing(c);
        if (st == PDF_OK) st = pdf_step(c, dt, steps_per_trial);
        int64_t n = 0;
        if (st == PDF_OK) st = pdf_kernel_time(c, kernel, &ms, &n);
        if (st == PDF_OK) st = pdf_sync(c);
        ms /= steps_per_trial;
        return st;
    };
    pdf_tuning t{};
    int st = PDF_OK;
    // particle kernel: resident blocks per SM
    {
        const int occ = particle_occupancy(c);
        int best = occ;
        double best_ms = 1e300;
        for (int per = 1; per <= occ && st == PDF_OK; ++per) {
            st = prepare_particle(c, per);
            double ms = 0;
            if (st == PDF_OK) st = trial(PDF_K_PARTICLE, ms);
            if (st == PDF_OK && ms < best_ms) { best_ms = ms; best = per; }
        }
        if (st == PDF_OK) st = prepare_particle(c, best);
        t.step_blocks_per_sm = best;
        t.ms_particle = best_ms;
    }
    // scatter block size
    if (st == PDF_OK) {
        const int cand[3] = {128, 256, 512};
        int best = 256;
        double best_ms = 1e300;
        for (int k = 0; k < 3 && st == PDF_OK; ++k) {
            c->scatter_threads = cand[k];
            double ms = 0;
            st = trial(PDF_K_SORT, ms);
            if (st == PDF_OK && ms < best_ms) { best_ms = ms; best = cand[k]; }
        }
        c->scatter_threads = best;
        t.scatter_threads = best;
        t.ms_sort = best_ms;
    }
    // CG block size (co-resident grids only)
    if (st == PDF_OK && c->p.wall_model == PDF_ELLIPTIC_RELAXATION) {
        const int cand[3] = {128, 160, 192};
        int best = 0;
        double best_ms = 1e300;
        for (int k = 0; k < 3 && st == PDF_OK; ++k) {
            if (prepare_elliptic(c, cand[k]) != PDF_OK) continue;  // not co-resident: skip
            double ms = 0;
            st = trial(PDF_K_ELLIPTIC, ms);
            if (st == PDF_OK && ms < best_ms) { best_ms = ms; best = cand[k]; }
        }
        if (st == PDF_OK) st = best ? prepare_elliptic(c, best) : prepare_elliptic(c, 0);
        t.cg_rows_per_block = c->fe_bs;
        t.ms_elliptic = best_ms;
    }
    // bins grid (FP32 state, 2x2x2 bins): it runs beside the field chain, so
    // the whole step's time decides
    t.bins_blocks_per_sm = -1;
    if (st == PDF_OK && c->prec != 0 && c->p.nb1 == 2 && c->p.nb2 == 2 && c->p.nb3 == 2) {
        const int cand[5] = {3, 4, 5, 6, 0};
        int best = c->bins_bps;
        double best_ms = 1e300;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        cudaError_t ce = cudaEventCreate(&ev[0]);
        if (ce == cudaSuccess) ce = cudaEventCreate(&ev[1]);
        if (ce != cudaSuccess) st = fail(c, PDF_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ce));
        for (int k = 0; k < 5 && st == PDF_OK; ++k) {
            c->bins_bps = cand[k];
            st = pdf_step(c, dt, 1);  // warm-up with the new grid
            if (st == PDF_OK) st = cudaEventRecord(ev[0], c->s) == cudaSuccess ? PDF_OK : PDF_ERR_CUDA;
            if (st == PDF_OK) st = pdf_step(c, dt, steps_per_trial);
            if (st == PDF_OK) st = cudaEventRecord(ev[1], c->s) == cudaSuccess ? PDF_OK : PDF_ERR_CUDA;
            if (st == PDF_OK) st = pdf_sync(c);
            float ms = 0.f;
            if (st == PDF_OK && cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) st = PDF_ERR_CUDA;
            if (st == PDF_OK) {
                t.ms_step_bins[k] = ms / steps_per_trial;
                if (t.ms_step_bins[k] < best_ms) { best_ms = t.ms_step_bins[k]; best = cand[k]; }
            }
        }
        c->bins_bps = best;
        t.bins_blocks_per_sm = best;
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    c->timing = timing;
    if (st == PDF_OK && out) *out = t;
    return st;
}

int pdf_apply_tuning(pdf_ctx* c, const pdf_tuning* t) {
    if (!c || !t) return PDF_ERR_ARG;
    const int sc = t->scatter_threads;
    if (t->step_blocks_per_sm < 1 || (sc != 128 && sc != 256 && sc != 512) || t->bins_blocks_per_sm < -1 ||
        (t->cg_rows_per_block != 0 && t->cg_rows_per_block != 128 && t->cg_rows_per_block != 160 &&
         t->cg_rows_per_block != 192))
        return fail(c, PDF_ERR_ARG, "pdf_apply_tuning: launch shape outside the tuned sets");
    int st = prepare_particle(c, t->step_blocks_per_sm);
    if (st != PDF_OK) return st;
    c->scatter_threads = sc;
    if (t->cg_rows_per_block && c->p.wall_model == PDF_ELLIPTIC_RELAXATION) {
        st = prepare_elliptic(c, t->cg_rows_per_block);
        if (st != PDF_OK) return st;
    }
    if (t->bins_blocks_per_sm >= 0) c->bins_bps = t->bins_blocks_per_sm;
    return PDF_OK;
}

}  // extern "C"
