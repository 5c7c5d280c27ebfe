// Checkpoint files (not in the paper): a fixed header that identifies the
// run, the state of qmc_get_state, and a 64-bit FNV-1a checksum (Fowler,
// Noll, Vo) of header and state.  Written to a temporary name, flushed to
// the storage device (fsync of the file), renamed, and the directory entry
// flushed too, so neither a crash nor a power loss leaves a truncated file
// under the final name or loses the previous checkpoint before the new one
// is on disk.  Host code only: no device calls.
#include <cstdio>
#include <cstring>
#include <fcntl.h>
#include <string>
#include <unistd.h>

#include "qmc.h"
#include "qmc_internal.cuh"

uint64_t qmc_fnv1a(const void *p, size_t n, uint64_t h)
{
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

static const uint64_t FNV_OFFSET = 0xcbf29ce484222325ull;

extern "C" {

int qmc_checkpoint_write(const char *path, const qmc_checkpoint_header *h, const double *state)
{
    if (!path || !h || !state || h->magic != QMC_CKPT_MAGIC || h->version != QMC_CKPT_VERSION)
        return QMC_ERR_ARG;
    const size_t nbytes = sizeof(double) * (size_t)h->n_doubles;
    uint64_t sum = qmc_fnv1a(h, sizeof *h, FNV_OFFSET);
    sum = qmc_fnv1a(state, nbytes, sum);
    std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid());
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return QMC_ERR_IO;
    bool ok = fwrite(h, sizeof *h, 1, f) == 1 &&
              (nbytes == 0 || fwrite(state, nbytes, 1, f) == 1) &&
              fwrite(&sum, sizeof sum, 1, f) == 1;
    ok = ok && fflush(f) == 0 && fsync(fileno(f)) == 0;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return QMC_ERR_IO;
    }
    // the rename itself is durable once the directory is flushed
    std::string dir(path);
    const size_t slash = dir.find_last_of('/');
    dir = slash == std::string::npos ? std::string(".") : dir.substr(0, slash ? slash : 1);
    const int dfd = open(dir.c_str(), O_RDONLY);
    if (dfd >= 0) {
        const int r = fsync(dfd);
        close(dfd);
        if (r != 0) return QMC_ERR_IO;
    }
    return QMC_OK;
}

int qmc_checkpoint_read_header(const char *path, qmc_checkpoint_header *h)
{
    if (!path || !h) return QMC_ERR_ARG;
    FILE *f = fopen(path, "rb");
    if (!f) return QMC_ERR_IO;
    bool ok = fread(h, sizeof *h, 1, f) == 1;
    fclose(f);
    if (!ok || h->magic != QMC_CKPT_MAGIC || h->version != QMC_CKPT_VERSION) return QMC_ERR_IO;
    return QMC_OK;
}

int qmc_checkpoint_read(const char *path, const qmc_checkpoint_header *expect, double *state,
                        size_t len)
{
    if (!path || !state) return QMC_ERR_ARG;
    qmc_checkpoint_header h;
    FILE *f = fopen(path, "rb");
    if (!f) return QMC_ERR_IO;
    int code = QMC_OK;
    if (fread(&h, sizeof h, 1, f) != 1 || h.magic != QMC_CKPT_MAGIC ||
        h.version != QMC_CKPT_VERSION) {
        code = QMC_ERR_IO;
    } else if (expect && memcmp(&h, expect, sizeof h) != 0) {
        code = QMC_ERR_ARG;   // another run's checkpoint
    } else if (len < h.n_doubles) {
        code = QMC_ERR_ARG;
    } else {
        const size_t nbytes = sizeof(double) * (size_t)h.n_doubles;
        uint64_t stored = 0, sum = qmc_fnv1a(&h, sizeof h, FNV_OFFSET);
        if ((nbytes && fread(state, nbytes, 1, f) != 1) || fread(&stored, sizeof stored, 1, f) != 1)
            code = QMC_ERR_IO;   // truncated
        else if (qmc_fnv1a(state, nbytes, sum) != stored)
            code = QMC_ERR_IO;   // corrupted
        else if (fgetc(f) != EOF)
            code = QMC_ERR_IO;   // trailing bytes: not a file this writer made
    }
    fclose(f);
    return code;
}

}  // extern "C"
