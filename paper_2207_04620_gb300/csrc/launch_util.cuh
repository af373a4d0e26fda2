// Launch helpers shared by the kernel files: grid sizing for the elementwise
// kernels, the per-class CUDA-event profiler hook and the launch check.
#pragma once
#include <string>

#include "internal.h"

namespace hx {
namespace {

inline int ew_blocks(int n, int per_thread) { return (n / per_thread + 255) / 256; }

// records a start/stop event pair around the launches in its scope when profiling
struct Timed {
    const LaunchCtx &c;
    Profiler::Rec r;
    Timed(const LaunchCtx &cc, int cls, double bytes) : c(cc)
    {
        if (!c.prof) return;
        r.cls = cls;
        r.bytes = bytes;
        r.a = c.prof->get();
        r.b = c.prof->get();
        cudaEventRecord(r.a, c.stream);
    }
    ~Timed()
    {
        if (!c.prof) return;
        cudaEventRecord(r.b, c.stream);
        c.prof->recs.push_back(r);
    }
};

inline void post(const LaunchCtx &c, int k = 1)
{
    if (c.launches) *c.launches += k;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error{HX_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e)};
}

} // namespace
} // namespace hx
