// gwas_stream: out-of-core GWAS from files through the C ABI (Algorithm 2, Section 3).
//
// The genotype file is read block by block by a reader thread into page-locked host
// buffers while earlier blocks are copied to the GPU and solved, so disk reads, host ->
// device copies and compute overlap as in the paper's double-buffered streaming; the
// relatedness matrix, covariates and phenotypes are read once and factored on the GPU.
//
// Inputs (raw little-endian arrays, column-major):
//   --phi FILE     n x n float64 (Phi; M = sigma2 (h Phi + (1-h) I)), or M itself with --m-given
//   --covar FILE   n x q float64 (X_L; q = p - 1 columns)
//   --pheno FILE   n x t float64 (Y)
//   --bed FILE     PLINK SNP-major .bed (magic 6c 1b 01, ceil(n/4) bytes per SNP; the
//                  dosage is the count of the first allele, missing calls give status 2)
//   --dosages FILE n bytes per SNP, int8 dosages {0,1,2}
// Outputs: PREFIX.b (m x t x p float64, SNP-major), PREFIX.wald (m x t float64),
// PREFIX.status (m uint8: 0 ok, 1 singular, 2 bad or missing genotype), written block by
// block, and one JSON line on stdout with the timings.
// Checkpoint / resume: with --checkpoint every completed block is flushed to disk and then
// recorded in PREFIX.progress (written to a temporary file and renamed, so it never claims
// more than is on disk); --resume continues a job from the blocks PREFIX.progress records
// (the job's sizes, formats, h, sigma2, input contents and genotype file must match);
// --max-blocks K stops cleanly after K new blocks (a time-sliced run; resume it later).
#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gwas.h"

namespace {

struct Args {
    int64_t n = 0, m = 0, m_blk = 16384;
    int q = 0, t = 1, limbs = 3, device = 0, readers = 2;
    double h = 0.4, sigma2 = 1.0;
    bool mixed = false, m_given = false, checkpoint = false, resume = false;
    int64_t max_blocks = -1;
    std::string phi, covar, pheno, bed, dosages, out;
};

[[noreturn]] void die(int code, const std::string& msg) {
    std::fprintf(stderr, "gwas_stream: %s\n", msg.c_str());
    std::exit(code);
}

void usage() {
    die(1, "usage: gwas_stream --n N --q Q [--t T] --phi F --covar F --pheno F "
           "(--bed F | --dosages F) --m M [--m-blk B] [--h H] [--sigma2 S] [--m-given] "
           "[--precision fp64|mixed] [--limbs L] [--device D] [--readers R] "
           "[--checkpoint] [--resume] [--max-blocks K] --out PREFIX");
}

Args parse(int argc, char** argv) {
    Args a;
    for (int i = 1; i < argc; ++i) {
        const std::string k = argv[i];
        auto val = [&]() -> std::string {
            if (i + 1 >= argc) usage();
            return argv[++i];
        };
        if (k == "--n") a.n = std::stoll(val());
        else if (k == "--q") a.q = std::stoi(val());
        else if (k == "--t") a.t = std::stoi(val());
        else if (k == "--m") a.m = std::stoll(val());
        else if (k == "--m-blk") a.m_blk = std::stoll(val());
        else if (k == "--h") a.h = std::stod(val());
        else if (k == "--sigma2") a.sigma2 = std::stod(val());
        else if (k == "--m-given") a.m_given = true;
        else if (k == "--limbs") a.limbs = std::stoi(val());
        else if (k == "--device") a.device = std::stoi(val());
        else if (k == "--readers") a.readers = std::stoi(val());
        else if (k == "--checkpoint") a.checkpoint = true;
        else if (k == "--resume") a.resume = a.checkpoint = true;
        else if (k == "--max-blocks") a.max_blocks = std::stoll(val()), a.checkpoint = true;
        else if (k == "--precision") {
            const std::string v = val();
            if (v == "mixed") a.mixed = true;
            else if (v != "fp64") usage();
        } else if (k == "--phi") a.phi = val();
        else if (k == "--covar") a.covar = val();
        else if (k == "--pheno") a.pheno = val();
        else if (k == "--bed") a.bed = val();
        else if (k == "--dosages") a.dosages = val();
        else if (k == "--out") a.out = val();
        else usage();
    }
    if (a.n < 1 || a.q < 1 || a.t < 1 || a.m < 1 || a.m_blk < 1 || a.readers < 1 ||
        a.readers > 8 || a.phi.empty() ||
        a.covar.empty() || a.pheno.empty() || a.out.empty() || a.bed.empty() == a.dosages.empty())
        usage();
    return a;
}

std::vector<double> read_f64(const std::string& path, size_t count) {
    std::vector<double> v(count);
    FILE* f = std::fopen(path.c_str(), "rb");
    if (!f) die(3, "cannot open " + path);
    const size_t got = std::fread(v.data(), sizeof(double), count, f);
    std::fclose(f);
    if (got != count) die(4, path + ": expected " + std::to_string(count) + " float64 values");
    return v;
}

void pwrite_all(int fd, const void* p, size_t bytes, off_t off, const std::string& what) {
    size_t done = 0;
    while (done < bytes) {
        const ssize_t w = ::pwrite(fd, (const char*)p + done, bytes - done, off + (off_t)done);
        if (w <= 0) die(5, "cannot write " + what);
        done += (size_t)w;
    }
}

// 64-bit checksum of an input array (FNV-1a over its 64-bit words): the progress file
// of a job records those of Phi, X_L and Y, so that a resume with other inputs is refused.
uint64_t checksum(const std::vector<double>& v) {
    uint64_t h = 1469598103934665603ull;
    for (double x : v) {
        uint64_t w;
        std::memcpy(&w, &x, sizeof w);
        h = (h ^ w) * 1099511628211ull;
    }
    return h;
}

// The job identity recorded with the progress: a resume must describe the same job --
// the same sizes, formats and model (h, sigma2, the inputs' contents) and the same
// genotype file (path and size).
std::string job_key(const Args& a, int64_t mblk, uint64_t sum_phi, uint64_t sum_xl,
                    uint64_t sum_y, const std::string& geno, int64_t geno_bytes) {
    char buf[512];
    std::snprintf(buf, sizeof buf,
                  "n=%lld m=%lld m_blk=%lld q=%d t=%d input=%s precision=%s limbs=%d h=%.17g "
                  "sigma2=%.17g m_given=%d phi=%016llx covar=%016llx pheno=%016llx "
                  "genotype_bytes=%lld genotypes=",
                  (long long)a.n, (long long)a.m, (long long)mblk, a.q, a.t,
                  a.bed.empty() ? "int8" : "bed", a.mixed ? "mixed" : "fp64", a.limbs, a.h,
                  a.sigma2, a.m_given ? 1 : 0, (unsigned long long)sum_phi,
                  (unsigned long long)sum_xl, (unsigned long long)sum_y, (long long)geno_bytes);
    std::string key = buf + geno;
    for (char& ch : key)
        if (ch == '\n' || ch == '\r') ch = '?';
    return key;
}

int64_t read_progress(const std::string& path, const std::string& key) {
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return 0;  // nothing done yet
    std::string s;
    for (int ch; (ch = std::fgetc(f)) != EOF && ch != '\n';) s.push_back((char)ch);
    std::fclose(f);
    const std::string head = "gwas_stream-progress " + key + " blocks=";
    if (s.compare(0, head.size(), head) != 0) die(6, path + " belongs to another job");
    return std::stoll(s.substr(head.size()));
}

void write_progress(const std::string& path, const std::string& key, int64_t blocks) {
    const std::string tmp = path + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) die(5, "cannot write " + tmp);
    std::fprintf(f, "gwas_stream-progress %s blocks=%lld\n", key.c_str(), (long long)blocks);
    std::fflush(f);
    ::fsync(::fileno(f));
    std::fclose(f);
    if (std::rename(tmp.c_str(), path.c_str()) != 0) die(5, "cannot update " + path);
}

void check(gwas_ctx* ctx, gwas_status st, const char* what) {
    if (st != GWAS_OK)
        die(2, std::string(what) + ": status " + std::to_string((int)st) + " " +
                   (ctx ? gwas_last_error(ctx) : ""));
}

// Fixed set of page-locked input buffers handed between the reader and the solver.
struct Ring {
    std::mutex mu;
    std::condition_variable cv;
    std::vector<int64_t> filled;  // block held by each buffer once read, -1 while free
    bool failed = false;
};

}  // namespace

int main(int argc, char** argv) {
    const Args a = parse(argc, argv);
    const int p = a.q + 1;
    const bool packed = !a.bed.empty();
    const int64_t per_snp = packed ? (a.n + 3) / 4 : a.n;
    const int64_t header = packed ? 3 : 0;
    const int fd = ::open(packed ? a.bed.c_str() : a.dosages.c_str(), O_RDONLY);
    if (fd < 0) die(3, "cannot open the genotype file");
    if (packed) {
        unsigned char magic[3] = {0, 0, 0};
        if (::pread(fd, magic, 3, 0) != 3 || magic[0] != 0x6c || magic[1] != 0x1b || magic[2] != 0x01)
            die(3, "not a SNP-major PLINK .bed file (magic 6c 1b 01)");
    }

    // setup: read Phi, X_L, Y; factor on the GPU
    const auto t_setup = std::chrono::steady_clock::now();
    const std::vector<double> phi = read_f64(a.phi, (size_t)(a.n * a.n));
    const std::vector<double> XL = read_f64(a.covar, (size_t)(a.n * a.q));
    const std::vector<double> Y = read_f64(a.pheno, (size_t)(a.n * a.t));
    gwas_opts o;
    gwas_default_opts(&o);
    o.precision = a.mixed ? GWAS_PREC_MIXED : GWAS_PREC_FP64;
    o.m_blk = (int)std::min<int64_t>(a.m_blk, a.m);
    o.n_limbs = a.limbs;
    o.device = a.device;
    gwas_ctx* ctx = nullptr;
    check(nullptr, gwas_init(a.n, p, a.t, &o, &ctx), "gwas_init");
    check(ctx, gwas_factor(ctx, phi.data(), a.m_given ? 0 : 1, a.h, a.sigma2, XL.data(), Y.data()),
          "gwas_factor");
    const double setup_s =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_setup).count();

    // streaming: NB page-locked input buffers and output slots; `readers` threads read
    // the blocks in turn (block blk by thread blk % readers) so that file reads overlap
    const int R = a.readers, NB = R + 2;
    const int64_t mblk = o.m_blk, nblk = (a.m + mblk - 1) / mblk;
    std::vector<void*> in(NB, nullptr), ob(NB, nullptr), ow(NB, nullptr), os(NB, nullptr);
    for (int k = 0; k < NB; ++k) {
        check(ctx, gwas_host_alloc((size_t)(per_snp * mblk), &in[k]), "gwas_host_alloc");
        check(ctx, gwas_host_alloc((size_t)(mblk * a.t * p * 8), &ob[k]), "gwas_host_alloc");
        check(ctx, gwas_host_alloc((size_t)(mblk * a.t * 8), &ow[k]), "gwas_host_alloc");
        check(ctx, gwas_host_alloc((size_t)mblk, &os[k]), "gwas_host_alloc");
    }
    // outputs, written block by block; blocks [b0, nblk) are this run's
    const std::string progress = a.out + ".progress";
    std::string key;
    if (a.checkpoint) {
        struct stat sb;
        if (::fstat(fd, &sb) != 0) die(3, "cannot stat the genotype file");
        key = job_key(a, mblk, checksum(phi), checksum(XL), checksum(Y),
                      packed ? a.bed : a.dosages, (int64_t)sb.st_size);
    }
    const int64_t b0 = a.resume ? read_progress(progress, key) : 0;
    if (b0 > nblk) die(6, progress + " records more blocks than the job has");
    const int64_t b_end = a.max_blocks >= 0 ? std::min(nblk, b0 + a.max_blocks) : nblk;
    const int oflags = O_RDWR | O_CREAT | (a.resume ? 0 : O_TRUNC);
    const int fb = ::open((a.out + ".b").c_str(), oflags, 0644);
    const int fw = ::open((a.out + ".wald").c_str(), oflags, 0644);
    const int fs = ::open((a.out + ".status").c_str(), oflags, 0644);
    if (fb < 0 || fw < 0 || fs < 0) die(5, "cannot open the output files " + a.out + ".*");
    if (a.checkpoint && !a.resume) write_progress(progress, key, 0);
    int64_t ok = 0;

    Ring ring;
    ring.filled.assign(NB, -1);
    // owner[k]: the last block collected from buffer k (initially k - NB, so that blocks
    // 0 .. NB-1 find their buffers free)
    std::vector<int64_t> owner(NB);
    for (int k = 0; k < NB; ++k) owner[k] = k - NB;
    std::vector<double> read_s(R, 0.0);
    // li = blk - b0 is the block's index in this run (buffers, owners, gwas_wait_block)
    auto read_loop = [&](int r) {
        for (int64_t li = r; b0 + li < b_end; li += R) {
            const int64_t blk = b0 + li;
            const int k = (int)(li % NB);
            {
                // buffer k is handed to block li once block li - NB has been collected
                std::unique_lock<std::mutex> lk(ring.mu);
                ring.cv.wait(lk, [&] { return owner[k] == li - NB || ring.failed; });
                if (ring.failed) return;
            }
            const int64_t mb = std::min(mblk, a.m - blk * mblk);
            const size_t bytes = (size_t)(per_snp * mb);
            const off_t off = (off_t)(header + blk * mblk * per_snp);
            const auto t0 = std::chrono::steady_clock::now();
            size_t done = 0;
            while (done < bytes) {
                const ssize_t got = ::pread(fd, (char*)in[k] + done, bytes - done, off + (off_t)done);
                if (got <= 0) break;
                done += (size_t)got;
            }
            read_s[r] += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            std::lock_guard<std::mutex> lk(ring.mu);
            if (done != bytes) ring.failed = true;
            else ring.filled[k] = li;
            ring.cv.notify_all();
            if (ring.failed) return;
        }
    };
    std::vector<std::thread> reader;
    for (int r = 0; r < R; ++r) reader.emplace_back(read_loop, r);
    auto join_readers = [&] {
        for (auto& th : reader) th.join();
    };

    static const int8_t PLINK[4] = {2, -1, 1, 0};  // 00 hom first, 01 missing, 10 het, 11 hom second
    const auto t0 = std::chrono::steady_clock::now();
    double wait_read_s = 0.0;
    auto collect = [&](int64_t li) {  // a completed block's outputs to the output files
        const int64_t blk = b0 + li;
        const int k = (int)(li % NB);
        check(ctx, gwas_wait_block(ctx, li, -1), "gwas_wait_block");
        const int64_t mb = std::min(mblk, a.m - blk * mblk);
        pwrite_all(fb, ob[k], (size_t)(mb * a.t * p * 8), (off_t)(blk * mblk * a.t * p * 8), a.out + ".b");
        pwrite_all(fw, ow[k], (size_t)(mb * a.t * 8), (off_t)(blk * mblk * a.t * 8), a.out + ".wald");
        pwrite_all(fs, os[k], (size_t)mb, (off_t)(blk * mblk), a.out + ".status");
        for (int64_t i = 0; i < mb; ++i) ok += (((const uint8_t*)os[k])[i] == 0);
        if (a.checkpoint) {  // on disk first, then recorded
            if (::fdatasync(fb) != 0 || ::fdatasync(fw) != 0 || ::fdatasync(fs) != 0)
                die(5, "cannot flush the output files");
            write_progress(progress, key, blk + 1);
        }
        std::lock_guard<std::mutex> lk(ring.mu);
        owner[k] = li;
        ring.filled[k] = -1;
        ring.cv.notify_all();
    };
    const int64_t nrun = b_end - b0;
    for (int64_t li = 0; li < nrun; ++li) {
        const int64_t blk = b0 + li;
        const int k = (int)(li % NB);
        {
            const auto tw = std::chrono::steady_clock::now();
            std::unique_lock<std::mutex> lk(ring.mu);
            ring.cv.wait(lk, [&] { return ring.filled[k] == li || ring.failed; });
            if (ring.failed) {
                lk.unlock();
                join_readers();
                die(4, "short read of the genotype file");
            }
            wait_read_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - tw).count();
        }
        const int64_t mb = std::min(mblk, a.m - blk * mblk);
        if (packed)
            check(ctx, gwas_solve_block_packed(ctx, (const uint8_t*)in[k], mb, PLINK, (double*)ob[k],
                                               (double*)ow[k], (uint8_t*)os[k]),
                  "gwas_solve_block_packed");
        else
            check(ctx, gwas_solve_block(ctx, (const int8_t*)in[k], mb, (double*)ob[k],
                                        (double*)ow[k], (uint8_t*)os[k]),
                  "gwas_solve_block");
        if (li >= NB - 1) collect(li - (NB - 1));
    }
    for (int64_t li = std::max<int64_t>(0, nrun - (NB - 1)); li < nrun; ++li) collect(li);
    join_readers();
    check(ctx, gwas_sync(ctx, -1), "gwas_sync");
    const double stream_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    ::close(fd);

    ::close(fb);
    ::close(fw);
    ::close(fs);
    const int64_t snps_run = std::min(a.m, b_end * mblk) - std::min(a.m, b0 * mblk);
    std::printf("{\"n\": %lld, \"m\": %lld, \"m_blk\": %lld, \"precision\": \"%s\", \"input\": \"%s\", "
                "\"first_block\": %lld, \"blocks_done\": %lld, \"blocks\": %lld, \"complete\": %s, "
                "\"setup_s\": %.3f, \"stream_s\": %.3f, \"snps_per_s\": %.1f, \"read_thread_s\": %.3f, "
                "\"solver_waited_for_reads_s\": %.3f, \"genotype_bytes\": %lld, \"status_ok\": %lld}\n",
                (long long)a.n, (long long)a.m, (long long)mblk, a.mixed ? "mixed" : "fp64",
                packed ? "bed" : "int8", (long long)b0, (long long)b_end, (long long)nblk,
                b_end == nblk ? "true" : "false", setup_s, stream_s,
                stream_s > 0 ? (double)snps_run / stream_s : 0.0,
                [&] { double t = 0; for (double v : read_s) t += v; return t; }(),
                wait_read_s, (long long)(per_snp * snps_run), (long long)ok);
    for (int k = 0; k < NB; ++k) {
        gwas_host_free(in[k]);
        gwas_host_free(ob[k]);
        gwas_host_free(ow[k]);
        gwas_host_free(os[k]);
    }
    gwas_finalize(ctx);
    return 0;
}
