// Per-kernel-class timing: CUDA events recorded around each launch on the
// launching stream, with the launch's algorithmic bytes.  Active only while a
// context has profiling enabled; read after the stream has been synchronised.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace spde {

enum ProfClass {
    PK_NOISE = 0,
    PK_SUMSQ,
    PK_RESIDUAL,
    PK_MINRES_A,
    PK_ALPHA,
    PK_MINRES_B,
    PK_MG_DOWN,
    PK_MG_COARSE,
    PK_MG_UP,
    PK_GIVENS,
    PK_MINRES_D,
    PK_ADD_CORR,
    PK_TRANSPOSE,
    PK_PROJECT,
    PK_FLUX,
    PK_SCHUR_APPLY,
    PK_CG_UPDATE,
    PK_OTHER,  // small bookkeeping launches (reductions, flags, init)
    PK_NCLASS
};

extern const char* const kProfNames[PK_NCLASS];

struct Profiler {
    bool on = false;
    int64_t launches[PK_NCLASS] = {};
    double ms[PK_NCLASS] = {};
    double bytes[PK_NCLASS] = {};
    struct Rec {
        int k;
        cudaEvent_t a, b;
        double bytes;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    Rec cur{};

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    void begin(int k, cudaStream_t st) {
        if (!on) return;
        cur = Rec{k, get(), get(), 0.0};
        cudaEventRecord(cur.a, st);
    }
    void end(cudaStream_t st, double b) {
        if (!on) return;
        cudaEventRecord(cur.b, st);
        cur.bytes = b;
        pending.push_back(cur);
    }
    // records not yet flushed: their byte counts can still be set once the
    // number of columns a launch really processed is known
    size_t mark() const { return pending.size(); }
    void scale(size_t i0, size_t i1, double f) {
        for (size_t i = i0; i < i1 && i < pending.size(); ++i) pending[i].bytes *= f;
    }
    void set_bytes(size_t i, double b) {
        if (i < pending.size()) pending[i].bytes = b;
    }
    // call after the stream is synchronised
    void flush() {
        for (auto& r : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
                launches[r.k] += 1;
                ms[r.k] += t;
                bytes[r.k] += r.bytes;
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
        cudaGetLastError();
    }
    void reset() {
        flush();
        for (int k = 0; k < PK_NCLASS; ++k) {
            launches[k] = 0;
            ms[k] = 0.0;
            bytes[k] = 0.0;
        }
    }
    ~Profiler() {
        flush();
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// profiler of the context whose call is running on this thread (or null)
extern thread_local Profiler* t_prof;

inline void prof_begin(int k, cudaStream_t st) {
    if (t_prof) t_prof->begin(k, st);
}
inline void prof_end(cudaStream_t st, double bytes) {
    if (t_prof) t_prof->end(st, bytes);
}

}  // namespace spde
