// isis_host.cu -- page-locked host buffers for the arrays a force step moves between host and device
// (particle positions in, forces out: 12 and 24 bytes per particle).
//
// The copy engines reach a page-locked host buffer through the host's I/O address translation, one entry per
// host page.  A 512^3 particle coordinate is 512 MiB: tens of thousands of base pages, and the copies slow down
// several times over when those translations are cold (observed between the solves of a step: 40 GB/s against
// the link's 190-210 GB/s).  So a buffer of at least one transparent huge page is mapped on a huge-page
// boundary and advised MADV_HUGEPAGE before its pages are first touched, then registered with the CUDA driver
// (cudaHostRegister); its translations are then one entry per huge page.  Smaller buffers, and kernels that
// grant no huge pages, get base pages, registered the same way.
#include <cuda_runtime.h>
#include <sys/mman.h>
#include <unistd.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <vector>

#include "isis.h"

namespace {

struct HostBuf {
  void* user;     // the address handed to the caller (huge-page aligned where huge pages are used)
  void* base;     // the mapping
  size_t maplen;  // its length
  size_t len;     // the registered length
};

std::mutex g_mu;
std::vector<HostBuf> g_bufs;

// The transparent huge page size the kernel reports (0 when it reports none).
size_t thp_size() {
  static const size_t hp = [] {
    unsigned long long v = 0;
    if (FILE* f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
      if (std::fscanf(f, "%llu", &v) != 1) v = 0;
      std::fclose(f);
    }
    return (size_t)v;
  }();
  return hp;
}

}  // namespace

extern "C" isis_status isis_host_alloc(size_t bytes, void** out) {
  if (!out || bytes == 0) return ISIS_EINVAL;
  *out = nullptr;
  const long pgs = sysconf(_SC_PAGESIZE);
  const size_t pg = pgs > 0 ? (size_t)pgs : 4096;
  const size_t hp = thp_size();
  const bool huge = hp > pg && hp % pg == 0 && bytes >= hp;
  const size_t unit = huge ? hp : pg;
  if (bytes > SIZE_MAX - 2 * unit) return ISIS_EINVAL;
  const size_t len = (bytes + unit - 1) / unit * unit;
  const size_t maplen = huge ? len + hp : len;  // slack for a huge-page aligned start
  void* base = mmap(nullptr, maplen, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (base == MAP_FAILED) return ISIS_ENOMEM;
  char* p = static_cast<char*>(base);
  if (huge) {
    p = reinterpret_cast<char*>(((uintptr_t)base + hp - 1) / hp * hp);
    (void)madvise(p, len, MADV_HUGEPAGE);  // advice: refused, the buffer is made of base pages
  }
  // first touch, one write per base page: where huge pages are granted each aligned huge page faults in whole
  for (size_t o = 0; o < len; o += pg) p[o] = 0;
  if (cudaHostRegister(p, len, cudaHostRegisterDefault) != cudaSuccess) {
    cudaGetLastError();
    munmap(base, maplen);
    return ISIS_ECUDA;
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_bufs.push_back({p, base, maplen, len});
  }
  *out = p;
  return ISIS_OK;
}

extern "C" isis_status isis_host_free(void* ptr) {
  if (!ptr) return ISIS_OK;
  HostBuf b{};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    size_t i = 0;
    while (i < g_bufs.size() && g_bufs[i].user != ptr) ++i;
    if (i == g_bufs.size()) return ISIS_EINVAL;
    b = g_bufs[i];
    g_bufs.erase(g_bufs.begin() + (long)i);
  }
  const cudaError_t e = cudaHostUnregister(b.user);
  if (e != cudaSuccess) cudaGetLastError();
  munmap(b.base, b.maplen);
  return e == cudaSuccess ? ISIS_OK : ISIS_ECUDA;
}
