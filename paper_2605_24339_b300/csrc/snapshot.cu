// snapshot.cu -- checkpoint and resume of a time-stepping context
// (ipc_save / ipc_load).  The paper has no counterpart: this is the
// checkpoint/resume subsystem of the library around the method.
//
// A snapshot holds what the next time step depends on beyond the scene and
// the parameters the context was created with: the pad state x and v (owned
// by the caller), the kinematic master's current pose, the number of steps
// taken, and -- when the context has a learned warm start -- its FP32
// parameters, Adam moments, Adam step and settings.  Everything else a step
// reads (grids, candidate buffers, the block pattern, tet data) is rebuilt
// from the scene, and every kernel is deterministic, so a context loaded from
// a snapshot continues bit for bit as the one that wrote it.
//
// File layout (little-endian, every field 8-byte aligned):
//   char     magic[8]   "GMCPSNAP"
//   uint32   version    1
//   uint32   flags      bit 0: a network follows
//   int64    n_vert, n_mvert, n_stri, n_tet, n_env
//   int32    precision, reserved
//   int64    step_count
//   double   x[n_vert][3], v[n_vert][3], xm[n_mvert][3]
//   if flags & 1:
//     double lr, beta1, beta2, eps, pos_scale, disp_scale, force_scale
//     int64  adam_step, n_param
//     float  P[n_param], M1[n_param], M2[n_param]   (padded to 8 bytes)
//   uint64   FNV-1a 64 of every byte before it
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gmcp_internal.cuh"

namespace gmcp {
namespace {

constexpr char kMagic[8] = {'G', 'M', 'C', 'P', 'S', 'N', 'A', 'P'};
constexpr uint32_t kVersion = 1;

struct Header {
    char magic[8];
    uint32_t version, flags;
    int64_t nv, nmv, ns, nt, n_env;
    int32_t precision, reserved;
    int64_t step_count;
};
static_assert(sizeof(Header) == 72, "snapshot header layout");

// FNV-1a, 64-bit (Fowler, Noll, Vo): offset basis and prime as published
struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    }
};

struct Writer {
    std::vector<unsigned char> buf;
    void put(const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        buf.insert(buf.end(), b, b + n);
        while (buf.size() % 8) buf.push_back(0);
    }
};

struct Reader {
    const std::vector<unsigned char>& buf;
    size_t at = 0;
    bool ok = true;
    bool get(void* p, size_t n) {
        const size_t pad = (n + 7) / 8 * 8;
        if (!ok || at + pad > buf.size()) return ok = false;
        memcpy(p, buf.data() + at, n);
        at += pad;
        return true;
    }
};

ipc_status snap_fail(Ctx& c, ipc_status st, const std::string& m) {
    c.err = m;
    return st;
}

}  // namespace
}  // namespace gmcp

using namespace gmcp;

extern "C" {

ipc_status ipc_save(ipc_ctx* ctx, const char* path, const double* x_dev, const double* v_dev) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx_of(ctx);
    if (!path || !x_dev || !v_dev) return snap_fail(c, IPC_ERR_ARG, "ipc_save: NULL path, x or v");
    if (c.joint) return snap_fail(c, IPC_ERR_ARG, "ipc_save: contexts with a master body are not supported");
    cudaError_t e = cudaSetDevice(c.device);
    const int64_t n3 = 3 * c.nv, m3 = 3 * c.nmv;
    std::vector<double> x(n3), v(n3), xm(m3);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x.data(), x_dev, sizeof(double) * n3, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v.data(), v_dev, sizeof(double) * n3, cudaMemcpyDeviceToHost, c.stream);
    // the master's current pose: the time stepper's copy once it exists, else the rest pose it starts from
    const double* xm_src = c.newton ? c.newton->xm.p : c.Y0.p;
    if (e == cudaSuccess && m3 > 0)
        e = cudaMemcpyAsync(xm.data(), xm_src, sizeof(double) * m3, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    WsState ws;
    if (e == cudaSuccess && c.ws) e = ws_state_get(c, &ws);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return snap_fail(c, IPC_ERR_CUDA, std::string("ipc_save: ") + cudaGetErrorString(e));
    }
    Header hd{};
    memcpy(hd.magic, kMagic, 8);
    hd.version = kVersion;
    hd.flags = c.ws ? 1u : 0u;
    hd.nv = c.nv; hd.nmv = c.nmv; hd.ns = c.ns; hd.nt = c.nt; hd.n_env = c.n_env;
    hd.precision = c.P.precision;
    hd.step_count = c.step_count;
    Writer w;
    w.put(&hd, sizeof(hd));
    w.put(x.data(), sizeof(double) * n3);
    w.put(v.data(), sizeof(double) * n3);
    w.put(xm.data(), sizeof(double) * m3);
    if (c.ws) {
        const double cfg[7] = {ws.lr, ws.beta1, ws.beta2, ws.eps, ws.pos_scale, ws.disp_scale, ws.force_scale};
        const int64_t ints[2] = {ws.step, (int64_t)ws.P.size()};
        w.put(cfg, sizeof(cfg));
        w.put(ints, sizeof(ints));
        w.put(ws.P.data(), sizeof(float) * ws.P.size());
        w.put(ws.M1.data(), sizeof(float) * ws.M1.size());
        w.put(ws.M2.data(), sizeof(float) * ws.M2.size());
    }
    Fnv f;
    f.add(w.buf.data(), w.buf.size());
    w.put(&f.h, sizeof(f.h));
    // write beside the target and rename, so a failed write never leaves a torn snapshot
    const std::string tmp = std::string(path) + ".tmp";
    FILE* fp = fopen(tmp.c_str(), "wb");
    if (!fp) return snap_fail(c, IPC_ERR_ARG, std::string("ipc_save: cannot open ") + tmp);
    const bool wrote = fwrite(w.buf.data(), 1, w.buf.size(), fp) == w.buf.size();
    const bool closed = fclose(fp) == 0;
    if (!wrote || !closed || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return snap_fail(c, IPC_ERR_ARG, std::string("ipc_save: write to ") + path + " failed");
    }
    return IPC_OK;
}

ipc_status ipc_load(ipc_ctx* ctx, const char* path, double* x_dev, double* v_dev, int64_t* step_count_host) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx_of(ctx);
    if (!path || !x_dev || !v_dev) return snap_fail(c, IPC_ERR_ARG, "ipc_load: NULL path, x or v");
    if (c.joint) return snap_fail(c, IPC_ERR_ARG, "ipc_load: contexts with a master body are not supported");
    std::vector<unsigned char> buf;
    {
        FILE* fp = fopen(path, "rb");
        if (!fp) return snap_fail(c, IPC_ERR_ARG, std::string("ipc_load: cannot open ") + path);
        unsigned char chunk[1 << 16];
        size_t got;
        while ((got = fread(chunk, 1, sizeof(chunk), fp)) > 0) buf.insert(buf.end(), chunk, chunk + got);
        fclose(fp);
    }
    if (buf.size() < sizeof(Header) + 8) return snap_fail(c, IPC_ERR_ARG, "ipc_load: file too short");
    {
        Fnv f;
        f.add(buf.data(), buf.size() - 8);
        uint64_t want;
        memcpy(&want, buf.data() + buf.size() - 8, 8);
        if (f.h != want) return snap_fail(c, IPC_ERR_ARG, "ipc_load: checksum mismatch (corrupt or truncated file)");
    }
    Reader r{buf};
    Header hd;
    r.get(&hd, sizeof(hd));
    if (memcmp(hd.magic, kMagic, 8) != 0) return snap_fail(c, IPC_ERR_ARG, "ipc_load: not a GMCP snapshot");
    if (hd.version != kVersion)
        return snap_fail(c, IPC_ERR_ARG, "ipc_load: snapshot version " + std::to_string(hd.version) +
                                              ", this library reads version " + std::to_string(kVersion));
    if (hd.nv != c.nv || hd.nmv != c.nmv || hd.ns != c.ns || hd.nt != c.nt || hd.n_env != c.n_env)
        return snap_fail(c, IPC_ERR_ARG, "ipc_load: the snapshot was written for a scene of other sizes");
    const int64_t n3 = 3 * c.nv, m3 = 3 * c.nmv;
    std::vector<double> x(n3), v(n3), xm(m3);
    r.get(x.data(), sizeof(double) * n3);
    r.get(v.data(), sizeof(double) * n3);
    r.get(xm.data(), sizeof(double) * m3);
    WsState ws;
    const bool has_ws = hd.flags & 1u;
    if (has_ws) {
        double cfg[7];
        int64_t ints[2];
        r.get(cfg, sizeof(cfg));
        r.get(ints, sizeof(ints));
        if (!r.ok || ints[1] != ws_param_count())
            return snap_fail(c, IPC_ERR_ARG, "ipc_load: the snapshot's network has another parameter count");
        ws.lr = cfg[0]; ws.beta1 = cfg[1]; ws.beta2 = cfg[2]; ws.eps = cfg[3];
        ws.pos_scale = cfg[4]; ws.disp_scale = cfg[5]; ws.force_scale = cfg[6];
        ws.step = ints[0];
        ws.P.resize(ints[1]); ws.M1.resize(ints[1]); ws.M2.resize(ints[1]);
        r.get(ws.P.data(), sizeof(float) * ints[1]);
        r.get(ws.M1.data(), sizeof(float) * ints[1]);
        r.get(ws.M2.data(), sizeof(float) * ints[1]);
    }
    if (!r.ok || r.at + 8 != buf.size()) return snap_fail(c, IPC_ERR_ARG, "ipc_load: malformed snapshot");
    // everything is read and checked: now change the context and the caller's arrays
    cudaError_t e = cudaSetDevice(c.device);
    if (e == cudaSuccess && c.nt > 0) e = newton_setup(c);
    if (e == cudaSuccess && has_ws && !c.ws) {
        ipc_ws_params wp{};
        wp.params_host = ws.P.data();
        wp.lr = ws.lr; wp.beta1 = ws.beta1; wp.beta2 = ws.beta2; wp.eps = ws.eps;
        wp.pos_scale = ws.pos_scale; wp.disp_scale = ws.disp_scale; wp.force_scale = ws.force_scale;
        const ipc_status st = ipc_ws_create(ctx, &wp);
        if (st != IPC_OK) return st;
    }
    if (e == cudaSuccess && has_ws) e = ws_state_set(c, ws);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x_dev, x.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v_dev, v.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess && c.newton && m3 > 0)
        e = cudaMemcpyAsync(c.newton->xm.p, xm.data(), sizeof(double) * m3, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return snap_fail(c, IPC_ERR_CUDA, std::string("ipc_load: ") + cudaGetErrorString(e));
    }
    c.step_count = hd.step_count;
    if (step_count_host) *step_count_host = hd.step_count;
    return IPC_OK;
}

}  // extern "C"
