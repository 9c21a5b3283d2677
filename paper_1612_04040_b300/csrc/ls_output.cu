// ls_output.cu -- overlapped output of phi snapshots (the output strategy of
// section 2: results are written while the computation goes on, by a worker
// that does nothing else).
//
// Here the worker is a host thread.  Every `every` steps the engine copies
// the current phi (bricked) into a free device snapshot slot on the compute
// stream (a device-to-device copy, ~0.2 ms for 512^3 FP32), a copy stream
// moves the slot to pinned host memory, and the writer thread turns it into
// a VTK XML file (.vts StructuredGrid with explicit point coordinates, as in
// the paper, or the compact .vti ImageData) while the GPU keeps stepping.
// When every slot is still in flight the engine waits for one (back
// pressure); the wait is counted.
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ls_ctx.cuh"

namespace lsk {

struct OutSlot {
    void* dev = nullptr;         // device snapshot (bricked)
    void* host = nullptr;        // pinned host copy
    cudaEvent_t copied = nullptr;  // snapshot taken (compute stream)
    cudaEvent_t landed = nullptr;  // host copy complete (copy stream)
    long long step = 0;
    bool busy = false;
};

struct Output {
    std::string prefix;
    int every = 1;
    int format = LS_OUTPUT_VTS;
    int device = 0;
    Inst in{};
    int prec = 0;
    size_t bytes = 0;
    cudaStream_t copy_stream = nullptr;
    std::vector<OutSlot> slots;
    std::deque<int> queue;
    std::mutex mu;
    std::condition_variable cv_work, cv_free;
    bool stop = false;
    std::thread writer;
    // statistics
    unsigned long long files = 0, written = 0;
    double write_s = 0.0, wait_s = 0.0;
    int status = LS_OK;
};

namespace {

// one z-plane of the snapshot in row-major order (x fastest)
template <typename T>
void plane_from_bricked(const T* b, const Inst& in, int z, T* out)
{
    const int tz = z >> 3, lz = z & 7;
    for (int y = 0; y < in.ny; ++y) {
        const int ty = y >> 3, ly = y & 7;
        for (int tx = 0; tx < in.tnx; ++tx) {
            const size_t t = ((size_t)tz * in.tny + ty) * in.tnx + tx;
            const T* src = b + t * TILE_PTS + (lz * 8 + ly) * 8;
            std::memcpy(out + (size_t)y * in.nx + tx * 8, src, 8 * sizeof(T));
        }
    }
}

template <typename T>
void plane_from_rowmajor(const T* a, const Inst& in, int z, T* out)
{
    std::memcpy(out, a + (size_t)z * in.nx * in.ny, (size_t)in.nx * in.ny * sizeof(T));
}

bool put(FILE* f, const void* p, size_t n) { return std::fwrite(p, 1, n, f) == n; }

// VTK XML, one piece, raw appended data (UInt64 byte counts).  Points (.vts)
// and the image origin (.vti) are the cell centres (i + 1/2) h.
template <typename T, typename Plane>
int write_vtk(const char* path, const Inst& in, int format, Plane plane, unsigned long long* nbytes)
{
    FILE* f = std::fopen(path, "wb");
    if (!f) return LS_EIO;
    const char* ty = sizeof(T) == 4 ? "Float32" : "Float64";
    const unsigned long long npts = (unsigned long long)in.nx * in.ny * in.nz;
    const unsigned long long phi_bytes = npts * sizeof(T);
    const unsigned long long pts_bytes = 3 * npts * sizeof(T);
    char head[2048];
    int len;
    if (format == LS_OUTPUT_VTS) {
        len = std::snprintf(
            head, sizeof(head),
            "<?xml version=\"1.0\"?>\n"
            "<VTKFile type=\"StructuredGrid\" version=\"1.0\" byte_order=\"LittleEndian\" "
            "header_type=\"UInt64\">\n"
            "  <StructuredGrid WholeExtent=\"0 %d 0 %d 0 %d\">\n"
            "    <Piece Extent=\"0 %d 0 %d 0 %d\">\n"
            "      <PointData Scalars=\"phi\">\n"
            "        <DataArray type=\"%s\" Name=\"phi\" NumberOfComponents=\"1\" format=\"appended\" "
            "offset=\"0\"/>\n"
            "      </PointData>\n"
            "      <Points>\n"
            "        <DataArray type=\"%s\" Name=\"Points\" NumberOfComponents=\"3\" format=\"appended\" "
            "offset=\"%llu\"/>\n"
            "      </Points>\n"
            "    </Piece>\n"
            "  </StructuredGrid>\n"
            "  <AppendedData encoding=\"raw\">\n_",
            in.nx - 1, in.ny - 1, in.nz - 1, in.nx - 1, in.ny - 1, in.nz - 1, ty, ty,
            (unsigned long long)(8 + phi_bytes));
    } else {
        const double o = 0.5 * in.h;
        len = std::snprintf(
            head, sizeof(head),
            "<?xml version=\"1.0\"?>\n"
            "<VTKFile type=\"ImageData\" version=\"1.0\" byte_order=\"LittleEndian\" "
            "header_type=\"UInt64\">\n"
            "  <ImageData WholeExtent=\"0 %d 0 %d 0 %d\" Origin=\"%.17g %.17g %.17g\" "
            "Spacing=\"%.17g %.17g %.17g\">\n"
            "    <Piece Extent=\"0 %d 0 %d 0 %d\">\n"
            "      <PointData Scalars=\"phi\">\n"
            "        <DataArray type=\"%s\" Name=\"phi\" NumberOfComponents=\"1\" format=\"appended\" "
            "offset=\"0\"/>\n"
            "      </PointData>\n"
            "    </Piece>\n"
            "  </ImageData>\n"
            "  <AppendedData encoding=\"raw\">\n_",
            in.nx - 1, in.ny - 1, in.nz - 1, o, o, o, in.h, in.h, in.h, in.nx - 1, in.ny - 1,
            in.nz - 1, ty);
    }
    bool ok = len > 0 && len < (int)sizeof(head) && put(f, head, (size_t)len);
    ok = ok && put(f, &phi_bytes, 8);
    std::vector<T> buf((size_t)3 * in.nx * in.ny);
    for (int z = 0; ok && z < in.nz; ++z) {
        plane(z, buf.data());
        ok = put(f, buf.data(), (size_t)in.nx * in.ny * sizeof(T));
    }
    if (ok && format == LS_OUTPUT_VTS) {
        ok = put(f, &pts_bytes, 8);
        for (int z = 0; ok && z < in.nz; ++z) {
            const T zc = (T)((z + 0.5) * in.h);
            size_t k = 0;
            for (int y = 0; y < in.ny; ++y) {
                const T yc = (T)((y + 0.5) * in.h);
                for (int x = 0; x < in.nx; ++x) {
                    buf[k++] = (T)((x + 0.5) * in.h);
                    buf[k++] = yc;
                    buf[k++] = zc;
                }
            }
            ok = put(f, buf.data(), k * sizeof(T));
        }
    }
    static const char tail[] = "\n  </AppendedData>\n</VTKFile>\n";
    ok = ok && put(f, tail, sizeof(tail) - 1);
    ok = (std::fclose(f) == 0) && ok;
    if (nbytes && ok) {
        *nbytes = (unsigned long long)len + 8 + phi_bytes + sizeof(tail) - 1 +
                  (format == LS_OUTPUT_VTS ? 8 + pts_bytes : 0);
    }
    return ok ? LS_OK : LS_EIO;
}

std::string file_name(const Output& O, long long step)
{
    char num[32];
    std::snprintf(num, sizeof(num), "%08lld", step);
    return O.prefix + num + (O.format == LS_OUTPUT_VTS ? ".vts" : ".vti");
}

void writer_loop(Output* O)
{
    cudaSetDevice(O->device);
    for (;;) {
        int j;
        {
            std::unique_lock<std::mutex> lk(O->mu);
            O->cv_work.wait(lk, [&] { return O->stop || !O->queue.empty(); });
            if (O->queue.empty()) return;  // stop requested and nothing left
            j = O->queue.front();
            O->queue.pop_front();
        }
        OutSlot& S = O->slots[(size_t)j];
        const auto t0 = std::chrono::steady_clock::now();
        int r = cudaEventSynchronize(S.landed) == cudaSuccess ? LS_OK : LS_ECUDA;
        unsigned long long nb = 0;
        if (r == LS_OK) {
            const std::string path = file_name(*O, S.step);
            const Inst in = O->in;
            if (O->prec == LS_FP32) {
                const float* b = (const float*)S.host;
                r = write_vtk<float>(path.c_str(), in, O->format,
                                     [&](int z, float* out) { plane_from_bricked(b, in, z, out); }, &nb);
            } else {
                const double* b = (const double*)S.host;
                r = write_vtk<double>(path.c_str(), in, O->format,
                                      [&](int z, double* out) { plane_from_bricked(b, in, z, out); }, &nb);
            }
        }
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        {
            std::lock_guard<std::mutex> lk(O->mu);
            O->write_s += dt;
            if (r == LS_OK) {
                O->files += 1;
                O->written += nb;
            } else if (O->status == LS_OK) {
                O->status = r;
            }
            S.busy = false;
        }
        O->cv_free.notify_all();
    }
}

}  // namespace

void output_free(Output* O)
{
    if (!O) return;
    {
        std::lock_guard<std::mutex> lk(O->mu);
        O->stop = true;
    }
    O->cv_work.notify_all();
    if (O->writer.joinable()) O->writer.join();
    for (OutSlot& S : O->slots) {
        if (S.dev) cudaFree(S.dev);
        if (S.host) cudaFreeHost(S.host);
        if (S.copied) cudaEventDestroy(S.copied);
        if (S.landed) cudaEventDestroy(S.landed);
    }
    if (O->copy_stream) cudaStreamDestroy(O->copy_stream);
    delete O;
}

}  // namespace lsk

using lsk::Output;

// after step number c->step_count: snapshot phi into a free slot and queue it
int ls_engine_output_after_step(ls_ctx* c, cudaStream_t s)
{
    Output* O = c->output;
    if (!O || c->step_count % O->every != 0) return LS_OK;
    int j = -1;
    {
        std::unique_lock<std::mutex> lk(O->mu);
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            for (size_t k = 0; k < O->slots.size(); ++k)
                if (!O->slots[k].busy) {
                    j = (int)k;
                    break;
                }
            if (j >= 0) break;
            O->cv_free.wait(lk);
        }
        O->wait_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        O->slots[(size_t)j].busy = true;
        O->slots[(size_t)j].step = c->step_count;
    }
    lsk::OutSlot& S = O->slots[(size_t)j];
    cudaError_t e = cudaMemcpyAsync(S.dev, c->phi[c->cur], O->bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(S.copied, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(O->copy_stream, S.copied, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S.host, S.dev, O->bytes, cudaMemcpyDeviceToHost, O->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(S.landed, O->copy_stream);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(O->mu);
        S.busy = false;
        return ls_engine_cuda_fail(e);
    }
    {
        std::lock_guard<std::mutex> lk(O->mu);
        O->queue.push_back(j);
    }
    O->cv_work.notify_one();
    return LS_OK;
}

extern "C" {

int ls_output_open(ls_ctx* c, const char* prefix, int every, int format, int slots)
{
    if (!c || !prefix || every < 1 || slots < 1 || slots > 8) return LS_EINVAL;
    if (format != LS_OUTPUT_VTS && format != LS_OUTPUT_VTI) return LS_EINVAL;
    if (c->batched || c->output) return c->output ? LS_ESTATE : LS_EINVAL;
    Output* O = new (std::nothrow) Output();
    if (!O) return LS_ENOMEM;
    O->prefix = prefix;
    O->every = every;
    O->format = format;
    O->in = c->insts[0];
    O->prec = c->prec;
    O->bytes = c->npts * c->esize;
    cudaGetDevice(&O->device);
    bool ok = cudaStreamCreateWithFlags(&O->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
    O->slots.resize((size_t)slots);
    for (lsk::OutSlot& S : O->slots) {
        ok = ok && cudaMalloc(&S.dev, O->bytes) == cudaSuccess;
        ok = ok && cudaMallocHost(&S.host, O->bytes) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&S.copied, cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&S.landed, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        lsk::output_free(O);
        return LS_ENOMEM;
    }
    O->writer = std::thread(lsk::writer_loop, O);
    c->output = O;
    c->output_every = every;
    c->graphs.clear();
    return LS_OK;
}

int ls_output_stats(ls_ctx* c, ls_output_report* st)
{
    if (!c || !st) return LS_EINVAL;
    std::memset(st, 0, sizeof(*st));
    Output* O = c->output;
    if (!O) return LS_OK;
    std::lock_guard<std::mutex> lk(O->mu);
    st->files = O->files;
    st->bytes = O->written;
    st->write_seconds = O->write_s;
    st->wait_seconds = O->wait_s;
    st->status = O->status;
    return LS_OK;
}

int ls_output_close(ls_ctx* c, ls_output_report* st)
{
    if (!c) return LS_EINVAL;
    Output* O = c->output;
    if (!O) {
        if (st) std::memset(st, 0, sizeof(*st));
        return LS_OK;
    }
    {
        std::lock_guard<std::mutex> lk(O->mu);
        O->stop = true;
    }
    O->cv_work.notify_all();
    if (O->writer.joinable()) O->writer.join();
    int r = O->status;
    if (st) {
        st->files = O->files;
        st->bytes = O->written;
        st->write_seconds = O->write_s;
        st->wait_seconds = O->wait_s;
        st->status = O->status;
    }
    lsk::output_free(O);
    c->output = nullptr;
    return r;
}

int ls_write_vtk(const char* path, const void* phi, int nx, int ny, int nz, double h, int precision,
                 int format)
{
    if (!path || !phi || nx < 1 || ny < 1 || nz < 1 || !(h > 0.0)) return LS_EINVAL;
    if (precision != LS_FP32 && precision != LS_FP64) return LS_EINVAL;
    if (format != LS_OUTPUT_VTS && format != LS_OUTPUT_VTI) return LS_EINVAL;
    Inst in{};
    in.nx = nx;
    in.ny = ny;
    in.nz = nz;
    in.h = h;
    if (precision == LS_FP32) {
        const float* a = (const float*)phi;
        return lsk::write_vtk<float>(path, in, format,
                                     [&](int z, float* out) { lsk::plane_from_rowmajor(a, in, z, out); },
                                     nullptr);
    }
    const double* a = (const double*)phi;
    return lsk::write_vtk<double>(path, in, format,
                                  [&](int z, double* out) { lsk::plane_from_rowmajor(a, in, z, out); },
                                  nullptr);
}

}  // extern "C"
