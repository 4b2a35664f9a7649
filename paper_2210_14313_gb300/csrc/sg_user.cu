// Run-time compilation of user integrands (sg_integrand_create, include/sg.h).
//
// The user's source and the library's generic fold kernel (sg_user_kernel.cuh,
// with the enumeration and reduction headers it includes) are compiled
// together by NVRTC for the current device and loaded with the runtime's
// library API (cudaLibraryLoadData), so the kernel is launched like any
// other.  NVRTC is opened with dlopen when first needed: the library does not
// depend on it unless user integrands are used.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/sg.h"
#include "sg_user.h"
#include "sg_user_sources.h"  // generated at build time: the headers below as strings

struct sg_integrand_s {
    int K = 0;
    int device = 0;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    std::string log;
};

namespace {

struct Nvrtc {
    bool ok = false;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

const Nvrtc &nvrtc() {
    static Nvrtc N;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so", "libnvrtc.so.13", "libnvrtc.so.12",
                               "/usr/local/cuda/lib64/libnvrtc.so", "/usr/local/cuda/targets/sbsa-linux/lib/libnvrtc.so",
                               "/usr/local/cuda/targets/x86_64-linux/lib/libnvrtc.so"};
        void *h = nullptr;
        for (const char *n : names)
            if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (!h) return;
        N.create = (decltype(N.create))dlsym(h, "nvrtcCreateProgram");
        N.compile = (decltype(N.compile))dlsym(h, "nvrtcCompileProgram");
        N.log_size = (decltype(N.log_size))dlsym(h, "nvrtcGetProgramLogSize");
        N.log = (decltype(N.log))dlsym(h, "nvrtcGetProgramLog");
        N.cubin_size = (decltype(N.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
        N.cubin = (decltype(N.cubin))dlsym(h, "nvrtcGetCUBIN");
        N.destroy = (decltype(N.destroy))dlsym(h, "nvrtcDestroyProgram");
        N.ok = N.create && N.compile && N.log_size && N.log && N.cubin_size && N.cubin && N.destroy;
    });
    return N;
}

}  // namespace

extern "C" sg_status sg_integrand_create(const char *source, int state_size, sg_integrand *out) {
    if (!source || !out) return SG_EINVAL;
    if (state_size < 1 || state_size > SG_USER_MAX_STATE) return SG_ERANGE;
    *out = nullptr;
    const Nvrtc &N = nvrtc();
    if (!N.ok) return SG_EUNSUPPORTED;
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
        return SG_ECUDA;
    sg_integrand_s *f = new sg_integrand_s();
    f->K = state_size;
    f->device = dev;
    std::string prog = std::string(source) + "\n#include \"sg_user_kernel.cuh\"\n";
    const char *hdr_src[] = {sg_src_internal, sg_src_fold_logic, sg_src_xsum, sg_src_reduce, sg_src_user_kernel};
    const char *hdr_names[] = {"sg_internal.h", "sg_fold_logic.h", "sg_xsum.h", "sg_reduce.cuh", "sg_user_kernel.cuh"};
    nvrtcProgram P = nullptr;
    if (N.create(&P, prog.c_str(), "sg_user.cu", 5, hdr_src, hdr_names) != NVRTC_SUCCESS) {
        delete f;
        return SG_ENOMEM;
    }
    const std::string arch = "--gpu-architecture=sm_" + std::to_string(major * 10 + minor);
    const std::string kdef = "-DSG_USER_K=" + std::to_string(state_size);
    const char *opts[] = {arch.c_str(), kdef.c_str(), "-std=c++17", "-default-device"};
    const nvrtcResult rc = N.compile(P, 4, opts);
    size_t ls = 0;
    N.log_size(P, &ls);
    if (ls > 1) {
        f->log.resize(ls);
        N.log(P, &f->log[0]);
        f->log.resize(ls - 1);
    }
    if (rc != NVRTC_SUCCESS) {
        N.destroy(&P);
        *out = f;  // keeps the log readable through sg_integrand_log
        return SG_EINVAL;
    }
    size_t cs = 0;
    N.cubin_size(P, &cs);
    std::vector<char> cubin(cs);
    N.cubin(P, cubin.data());
    N.destroy(&P);
    if (cudaLibraryLoadData(&f->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
        cudaLibraryGetKernel(&f->kern, f->lib, "sg_user_fold") != cudaSuccess) {
        cudaGetLastError();
        if (f->lib) cudaLibraryUnload(f->lib);
        delete f;
        return SG_ECUDA;
    }
    *out = f;
    return SG_OK;
}

extern "C" sg_status sg_integrand_destroy(sg_integrand f) {
    if (!f) return SG_OK;
    if (f->lib) cudaLibraryUnload(f->lib);
    delete f;
    return SG_OK;
}

extern "C" sg_status sg_integrand_log(sg_integrand f, char *buf, size_t cap, size_t *len) {
    if (!f) return SG_EINVAL;
    if (len) *len = f->log.size();
    if (buf && cap) {
        const size_t n = f->log.size() < cap - 1 ? f->log.size() : cap - 1;
        memcpy(buf, f->log.data(), n);
        buf[n] = 0;
    }
    return SG_OK;
}

bool sg_integrand_kernel(sg_integrand f, cudaKernel_t *kern, int *K, int *device) {
    if (!f || !f->kern) return false;
    *kern = f->kern;
    *K = f->K;
    *device = f->device;
    return true;
}
