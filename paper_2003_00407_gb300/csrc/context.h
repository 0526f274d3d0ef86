// The library context (opaque to callers): device, last error, named device workspaces grown on
// demand, pinned readback words.
#pragma once
#include <map>
#include <string>

struct dgdft_ctx {
  int device = 0;
  std::string err;
  std::map<std::string, std::pair<void*, size_t>> bufs;
  bool tw_ready = false;
  int* h_active = nullptr;  // pinned readback: active-element count and the max residual
};
