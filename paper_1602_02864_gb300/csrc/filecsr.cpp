// filecsr.cpp -- the sparse matrix in a file: the paper's semi-external layout.
//
// Section 3.1 keeps vertex-sized state in memory and the edge-sized sparse
// matrix on SSDs, and streams the matrix for every multiplication.  A handle
// made by spmm_create_file keeps the row pointers (8 bytes per vertex) in
// pinned host memory and the plan in HBM, and reads the column indices and
// values (4 + v bytes per edge) from the file in blocks on every apply.
//
// File layout (little-endian; every section starts on a 4096-byte boundary so
// the sections can be read with O_DIRECT):
//   offset 0     header: "SPMMCSR1", int64 n_rows, n_cols, nnz, int32 vtype
//                (-1 pattern, else spmm_dtype), int32 0, int64 offsets of the
//                row pointers, column indices and values (0 if none)
//   off_rp       int64 row_ptr[n_rows + 1]
//   off_ci       int32 col_idx[nnz]
//   off_val      values[nnz] of vtype (absent for a pattern matrix)
#include <errno.h>
#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace spmm {

namespace {

constexpr char kMagic[8] = {'S', 'P', 'M', 'M', 'C', 'S', 'R', '1'};

struct Header {
    char magic[8];
    int64_t n_rows, n_cols, nnz;
    int32_t vtype, zero;
    int64_t off_rp, off_ci, off_val;
};

int64_t align_up(int64_t x) { return (x + kFileAlign - 1) / kFileAlign * kFileAlign; }

size_t vbytes(int32_t vtype) { return vtype < 0 ? 0 : (vtype == SPMM_F32 ? 4 : 2); }

bool write_all(int fd, const void* p, size_t n) {
    const char* c = static_cast<const char*>(p);
    while (n > 0) {
        const ssize_t w = ::write(fd, c, n);
        if (w < 0) {
            if (errno == EINTR) continue;
            return false;
        }
        c += w;
        n -= (size_t)w;
    }
    return true;
}

bool pad_to(int fd, int64_t* pos, int64_t target) {
    static const char zeros[kFileAlign] = {};
    while (*pos < target) {
        const size_t n = (size_t)std::min<int64_t>(target - *pos, kFileAlign);
        if (!write_all(fd, zeros, n)) return false;
        *pos += (int64_t)n;
    }
    return true;
}

}  // namespace

// Read [off, off + len) of the file into buf (which has room for the range
// widened to kFileAlign boundaries) with up to `threads` parallel preads.
// Returns a pointer to byte `off` inside buf, or nullptr (error text in *err).
// If n_cols_check > 0 the range holds int32 column indices: each reader
// checks its whole elements against [0, n_cols_check).
const char* file_read_range(int fd, bool direct, int64_t off, int64_t len, char* buf, int threads,
                            int64_t n_cols_check, std::string* err) {
    if (len == 0) return buf;
    const int64_t a0 = direct ? off / kFileAlign * kFileAlign : off;
    const int64_t a1 = direct ? align_up(off + len) : off + len;
    const int64_t total = a1 - a0;
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(threads, total / (1 << 20)));
    // pieces on kFileAlign boundaries
    std::vector<int64_t> cut((size_t)nt + 1);
    for (int i = 0; i <= nt; ++i)
        cut[(size_t)i] = i == nt ? total : std::min<int64_t>(total, (total * i / nt) / kFileAlign * kFileAlign);
    std::atomic<int> failed{0};
    std::atomic<int64_t> bad_at{-1};
    std::atomic<int> err_no{0};
    auto work = [&](int i) {
        int64_t p = cut[(size_t)i];
        const int64_t end = cut[(size_t)i + 1];
        while (p < end) {
            const ssize_t r = ::pread(fd, buf + p, (size_t)(end - p), (off_t)(a0 + p));
            if (r < 0) {
                if (errno == EINTR) continue;
                err_no.store(errno);
                failed.store(1);
                return;
            }
            if (r == 0) {   // the file ends early
                failed.store(2);
                return;
            }
            p += r;
        }
        if (n_cols_check > 0) {
            // whole int32 elements of [off, off + len) that start in this piece
            const int64_t lo = std::max<int64_t>(cut[(size_t)i] + a0, off), hi = std::min<int64_t>(end + a0, off + len);
            int64_t e0 = (lo - off + 3) / 4, e1 = (hi - off + 3) / 4;
            const int32_t* col = reinterpret_cast<const int32_t*>(buf + (off - a0));
            for (int64_t e = e0; e < e1; ++e)
                if (col[e] < 0 || (int64_t)col[e] >= n_cols_check) {
                    bad_at.store(e);
                    break;
                }
        }
    };
    if (nt == 1) {
        work(0);
    } else {
        std::vector<std::thread> pool;
        pool.reserve((size_t)nt);
        for (int i = 0; i < nt; ++i) pool.emplace_back(work, i);
        for (auto& t : pool) t.join();
    }
    if (failed.load() == 1) {
        *err = std::string("read failed: ") + std::strerror(err_no.load());
        return nullptr;
    }
    if (failed.load() == 2) {
        *err = "the file is shorter than its header says";
        return nullptr;
    }
    if (bad_at.load() >= 0) {
        *err = "column index out of range at element " + std::to_string(bad_at.load()) + " of the block";
        return nullptr;
    }
    return buf + (off - a0);
}

int file_open(const char* path, bool direct, FileCSR* f) {
    *f = FileCSR{};
    const int fd = ::open(path, O_RDONLY | (direct ? O_DIRECT : 0));
    if (fd < 0) {
        const int en = errno;
        set_error(std::string("spmm_create_file: cannot open ") + path + ": " + std::strerror(en));
        return (direct && en == EINVAL) ? SPMM_ERR_UNSUPPORTED : SPMM_ERR_IO;
    }
    // the header through a buffered descriptor (O_DIRECT wants aligned buffers)
    Header h;
    const int hfd = ::open(path, O_RDONLY);
    const bool ok = hfd >= 0 && ::pread(hfd, &h, sizeof(h), 0) == (ssize_t)sizeof(h);
    struct stat st;
    const bool ok_stat = hfd >= 0 && ::fstat(hfd, &st) == 0;
    if (hfd >= 0) ::close(hfd);
    if (!ok || !ok_stat || std::memcmp(h.magic, kMagic, 8) != 0) {
        ::close(fd);
        set_error(std::string("spmm_create_file: ") + path + " is not an SPMMCSR1 file");
        return SPMM_ERR_FORMAT;
    }
    const size_t vb = vbytes(h.vtype);
    const bool shape_ok = h.n_rows >= 0 && h.n_rows < ((int64_t)1 << 31) && h.n_cols >= 1 &&
                          h.n_cols < ((int64_t)1 << 31) && h.nnz >= 0 &&
                          (h.vtype == -1 || h.vtype == SPMM_F32 || h.vtype == SPMM_BF16 || h.vtype == SPMM_F16);
    const bool offs_ok = shape_ok && h.off_rp >= (int64_t)sizeof(Header) && h.off_rp % kFileAlign == 0 &&
                         h.off_ci % kFileAlign == 0 && h.off_ci >= h.off_rp + (h.n_rows + 1) * 8 &&
                         (vb == 0 || (h.off_val % kFileAlign == 0 && h.off_val >= h.off_ci + h.nnz * 4)) &&
                         (int64_t)st.st_size >= (vb ? h.off_val + h.nnz * (int64_t)vb : h.off_ci + h.nnz * 4);
    if (!offs_ok) {
        ::close(fd);
        set_error(std::string("spmm_create_file: bad header or truncated file: ") + path);
        return SPMM_ERR_FORMAT;
    }
    f->fd = fd;
    f->direct = direct;
    f->n_rows = h.n_rows;
    f->n_cols = h.n_cols;
    f->nnz = h.nnz;
    f->vtype = h.vtype;
    f->off_rp = h.off_rp;
    f->off_ci = h.off_ci;
    f->off_val = h.off_val;
    return SPMM_OK;
}

}  // namespace spmm

using namespace spmm;

extern "C" int spmm_write_csr_file(const char* path, int64_t n_rows, int64_t n_cols, int64_t nnz,
                                   const int64_t* row_ptr, const int32_t* col_idx, const void* values,
                                   spmm_dtype vtype) {
    if (!path || !row_ptr || (nnz > 0 && !col_idx) || n_rows < 0 || n_rows >= ((int64_t)1 << 31) || n_cols < 1 ||
        n_cols >= ((int64_t)1 << 31) || nnz < 0) {
        set_error("spmm_write_csr_file: bad shape or NULL array");
        return SPMM_ERR_ARG;
    }
    if (values && vtype != SPMM_F32 && vtype != SPMM_BF16 && vtype != SPMM_F16) {
        set_error("spmm_write_csr_file: values must be F32, BF16 or F16");
        return SPMM_ERR_ARG;
    }
    if (row_ptr[0] != 0 || row_ptr[n_rows] != nnz) {
        set_error("spmm_write_csr_file: row_ptr[0] must be 0 and row_ptr[n_rows] must be nnz");
        return SPMM_ERR_FORMAT;
    }
    for (int64_t i = 0; i < n_rows; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) {
            set_error("spmm_write_csr_file: row_ptr decreases at row " + std::to_string(i));
            return SPMM_ERR_FORMAT;
        }
    for (int64_t p = 0; p < nnz; ++p)
        if (col_idx[p] < 0 || (int64_t)col_idx[p] >= n_cols) {
            set_error("spmm_write_csr_file: column index out of range at entry " + std::to_string(p));
            return SPMM_ERR_FORMAT;
        }
    const int32_t vt = values ? (int32_t)vtype : -1;
    const size_t vb = vbytes(vt);
    Header h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, 8);
    h.n_rows = n_rows;
    h.n_cols = n_cols;
    h.nnz = nnz;
    h.vtype = vt;
    h.off_rp = kFileAlign;
    h.off_ci = align_up(h.off_rp + (n_rows + 1) * 8);
    h.off_val = vb ? align_up(h.off_ci + nnz * 4) : 0;
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid());
    const int fd = ::open(tmp.c_str(), O_WRONLY | O_CREAT | O_TRUNC, 0644);
    if (fd < 0) {
        set_error(std::string("spmm_write_csr_file: cannot create ") + tmp + ": " + std::strerror(errno));
        return SPMM_ERR_IO;
    }
    int64_t pos = 0;
    bool ok = write_all(fd, &h, sizeof(h)) && ((pos = sizeof(h)), pad_to(fd, &pos, h.off_rp)) &&
              write_all(fd, row_ptr, (size_t)(n_rows + 1) * 8) && ((pos += (n_rows + 1) * 8), pad_to(fd, &pos, h.off_ci)) &&
              write_all(fd, col_idx, (size_t)nnz * 4);
    pos += nnz * 4;
    if (ok && vb) ok = pad_to(fd, &pos, h.off_val) && write_all(fd, values, (size_t)nnz * vb) && ((pos += nnz * (int64_t)vb), true);
    if (ok) ok = pad_to(fd, &pos, align_up(pos));   // whole blocks at the end, for O_DIRECT readers
    ok = (::close(fd) == 0) && ok;
    if (!ok || ::rename(tmp.c_str(), path) != 0) {
        const int en = errno;
        ::unlink(tmp.c_str());
        set_error(std::string("spmm_write_csr_file: write failed: ") + std::strerror(en));
        return SPMM_ERR_IO;
    }
    return SPMM_OK;
}
