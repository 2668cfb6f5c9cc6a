// Disk -> pinned host memory, ahead of the GPU (Sec. 3.1: the data is
// streamed from disk to main memory to the GPU; the paper keeps three host
// buffers so that a disk read, a host->GPU copy and the CPU's own work can
// proceed at once).  A reader thread fills a ring of `depth` pinned buffers
// with consecutive blocks of a file (pread, 64-bit offsets); each block is
// read by a pool of worker threads in parallel byte ranges (one thread's
// copies out of the page cache run at a few GB/s, far below the host->GPU
// link); the consumer takes blocks in order and hands each back once its
// host->GPU copy is done.  Every wait is bounded; read errors and short reads
// surface as GWAS_ERR_IO.
#include <cuda_runtime.h>
#include <fcntl.h>
#include <unistd.h>

#include <algorithm>
#include <cerrno>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gwas_internal.cuh"

struct gwas_reader {
  int fd = -1;
  int64_t offset = 0, block_bytes = 0, nblocks = 0, last_bytes = 0;
  int depth = 0;
  std::vector<void*> buf;      // pinned
  bool own_buffers = true;     // false: the caller's buffers, kept on close
  std::vector<int64_t> bytes;  // bytes held by each buffer
  // slot s holds block b when b % depth == s; `filled` counts blocks read,
  // `taken` blocks handed to the consumer, `released` blocks given back
  int64_t filled = 0, taken = 0, released = 0;
  int error = 0;  // GWAS_ERR_IO after a failed or short read
  std::string detail;
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv;
  std::thread th;
  // the worker pool: job `job` asks each worker k for its part of one block
  std::vector<std::thread> workers;
  std::condition_variable wcv;
  int64_t job = 0;          // jobs posted
  char* job_dst = nullptr;  // the block's buffer
  int64_t job_off = 0, job_bytes = 0;
  int pending = 0;          // workers still reading the current job
};

namespace {

constexpr int64_t kPartAlign = 1 << 20;  // workers read whole MiB ranges

// Worker k reads its range of each posted block.
void worker_loop(gwas_reader* r, int k) {
  const int nw = (int)r->workers.size();
  int64_t seen = 0;
  while (true) {
    char* dst;
    int64_t off, bytes;
    {
      std::unique_lock<std::mutex> lk(r->mu);
      r->wcv.wait(lk, [&] { return r->job > seen || r->stop; });
      if (r->job == seen) return;  // stopped with no job left: a posted job is always finished
      seen = r->job;
      dst = r->job_dst;
      off = r->job_off;
      bytes = r->job_bytes;
    }
    int64_t part = (bytes + nw - 1) / nw;
    part = (part + kPartAlign - 1) / kPartAlign * kPartAlign;
    const int64_t lo = std::min<int64_t>(bytes, k * part), hi = std::min<int64_t>(bytes, lo + part);
    int64_t got = lo;
    std::string err;
    while (got < hi) {
      const ssize_t n = pread(r->fd, dst + got, (size_t)(hi - got), (off_t)(off + got));
      if (n < 0 && errno == EINTR) continue;
      if (n <= 0) {
        err = n < 0 ? std::string("read failed: ") + strerror(errno) : "file shorter than the requested blocks";
        break;
      }
      got += n;
    }
    std::lock_guard<std::mutex> lk(r->mu);
    if (!err.empty() && !r->error) {
      r->error = GWAS_ERR_IO;
      r->detail = err;
    }
    if (--r->pending == 0) r->cv.notify_all();
  }
}

void reader_loop(gwas_reader* r) {
  for (int64_t b = 0; b < r->nblocks; ++b) {
    {
      std::unique_lock<std::mutex> lk(r->mu);
      r->cv.wait(lk, [&] { return r->stop || b - r->released < r->depth; });
      if (r->stop) return;
    }
    const int s = (int)(b % r->depth);
    const int64_t want = (b == r->nblocks - 1) ? r->last_bytes : r->block_bytes;
    std::unique_lock<std::mutex> lk(r->mu);
    r->job_dst = static_cast<char*>(r->buf[s]);
    r->job_off = r->offset + b * r->block_bytes;
    r->job_bytes = want;
    r->pending = (int)r->workers.size();
    ++r->job;
    r->wcv.notify_all();
    // workers finish their reads whatever happens (stop is only set once they are idle)
    r->cv.wait(lk, [&] { return r->pending == 0; });
    if (r->error) {
      r->cv.notify_all();
      return;
    }
    r->bytes[s] = want;
    r->filled = b + 1;
    r->cv.notify_all();
  }
}

int reader_threads() {
  const unsigned hc = std::thread::hardware_concurrency();
  return hc >= 16 ? 8 : (hc >= 4 ? (int)hc / 2 : 1);
}

void start_threads(gwas_reader* r) {
  const int nw = reader_threads();
  r->workers.reserve(nw);
  for (int k = 0; k < nw; ++k) r->workers.emplace_back();
  for (int k = 0; k < nw; ++k) r->workers[k] = std::thread(worker_loop, r, k);
  r->th = std::thread(reader_loop, r);
}

}  // namespace

namespace gwas {

// As gwas_reader_open with `depth` caller-owned pinned buffers of at least
// block_bytes each (not freed on close): repeated streams reuse one pinned pool.
int reader_open_with(gwas_reader** out, const char* path, int64_t offset, int64_t block_bytes, int64_t nblocks,
                     int64_t last_bytes, int depth, void* const* buffers) {
  if (!out || !path || !buffers || offset < 0 || block_bytes < 1 || nblocks < 0 || depth < 2 || last_bytes < 0 ||
      last_bytes > block_bytes)
    return GWAS_ERR_ARG;
  *out = nullptr;
  gwas_reader* r = new gwas_reader;
  r->offset = offset;
  r->block_bytes = block_bytes;
  r->nblocks = nblocks;
  r->last_bytes = last_bytes ? last_bytes : block_bytes;
  r->depth = depth;
  r->fd = open(path, O_RDONLY);
  if (r->fd < 0) {
    delete r;
    return GWAS_ERR_IO;
  }
  r->buf.assign(buffers, buffers + depth);
  r->bytes.assign(depth, 0);
  r->own_buffers = false;
  start_threads(r);
  *out = r;
  return GWAS_OK;
}

}  // namespace gwas

extern "C" {

int gwas_reader_open(gwas_reader** out, const char* path, int64_t offset, int64_t block_bytes, int64_t nblocks,
                     int64_t last_bytes, int depth) {
  if (!out || !path || offset < 0 || block_bytes < 1 || nblocks < 0 || depth < 2 || last_bytes < 0 ||
      last_bytes > block_bytes)
    return GWAS_ERR_ARG;
  *out = nullptr;
  gwas_reader* r = new gwas_reader;
  r->offset = offset;
  r->block_bytes = block_bytes;
  r->nblocks = nblocks;
  r->last_bytes = last_bytes ? last_bytes : block_bytes;
  r->depth = depth;
  r->fd = open(path, O_RDONLY);
  if (r->fd < 0) {
    delete r;
    return GWAS_ERR_IO;
  }
  r->buf.assign(depth, nullptr);
  r->bytes.assign(depth, 0);
  for (auto& p : r->buf) {
    if (cudaMallocHost(&p, (size_t)block_bytes) != cudaSuccess) {
      cudaGetLastError();
      for (auto* q : r->buf) cudaFreeHost(q);
      close(r->fd);
      delete r;
      return GWAS_ERR_NOMEM;
    }
  }
  start_threads(r);
  *out = r;
  return GWAS_OK;
}

// The next block in file order: *buf (pinned) and *bytes; waits at most
// timeout_ms.  The buffer stays valid until gwas_reader_release.
int gwas_reader_next(gwas_reader* r, const void** buf, int64_t* bytes, int timeout_ms) {
  if (!r || !buf || !bytes) return GWAS_ERR_ARG;
  std::unique_lock<std::mutex> lk(r->mu);
  if (r->taken >= r->nblocks) return GWAS_ERR_ARG;
  const bool ok = r->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                 [&] { return r->error || r->filled > r->taken; });
  if (r->filled > r->taken) {
    const int s = (int)(r->taken % r->depth);
    *buf = r->buf[s];
    *bytes = r->bytes[s];
    ++r->taken;
    return GWAS_OK;
  }
  if (r->error) return r->error;
  return ok ? GWAS_ERR_IO : GWAS_ERR_TIMEOUT;
}

// Gives the oldest taken buffer back to the reader (its copy must be done).
int gwas_reader_release(gwas_reader* r) {
  if (!r) return GWAS_ERR_ARG;
  std::lock_guard<std::mutex> lk(r->mu);
  if (r->released >= r->taken) return GWAS_ERR_ARG;
  ++r->released;
  r->cv.notify_all();
  return GWAS_OK;
}

const char* gwas_reader_error_detail(const gwas_reader* r) { return r ? r->detail.c_str() : ""; }

void gwas_reader_close(gwas_reader* r) {
  if (!r) return;
  {
    std::lock_guard<std::mutex> lk(r->mu);
    r->stop = true;
    r->cv.notify_all();
  }
  if (r->th.joinable()) r->th.join();  // the reader thread returns between jobs
  {
    std::lock_guard<std::mutex> lk(r->mu);
    r->wcv.notify_all();
  }
  for (auto& w : r->workers)
    if (w.joinable()) w.join();
  if (r->own_buffers)
    for (auto* p : r->buf) cudaFreeHost(p);
  if (r->fd >= 0) close(r->fd);
  delete r;
}

}  // extern "C"
