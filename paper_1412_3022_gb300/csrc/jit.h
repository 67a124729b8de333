// Run-time compilation of generated device code (jit.cpp).
#pragma once
#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

#include "code.h"

namespace pmrc {

// Whether NVRTC could be loaded in this process.
bool jit_available();

// Compiles CUDA source for sm_103a into a cubin (kEUnsupported with the
// compiler log in err when NVRTC is missing or the source does not build).
// Cubins are kept on disk under a hash of the source, the options and the
// NVRTC version, and a later compilation of the same source (in this or
// another process) reads the file instead.  The directory is
// $PMRC_KERNEL_CACHE when set (empty, "0" or "off" turns the cache off),
// else $XDG_CACHE_HOME/pmrc or $HOME/.cache/pmrc; cache files that cannot be
// read or written are ignored.
int jit_compile(const std::string &src, const char *kernel_name, std::vector<char> &cubin,
                std::string &err);

// Runs fn on one of a few background threads (compilations that must not
// hold up the call that asked for them).  Jobs still queued when the
// process exits are dropped; a job already running is waited for, so no
// compilation is left inside NVRTC while the process tears down.
void jit_background(std::function<void()> fn);

// Loads a cubin as a CUDA library and finds its kernel `kernel_name`.
int jit_load(const std::vector<char> &cubin, const char *kernel_name, cudaLibrary_t *lib,
             cudaKernel_t *fn, std::string &err);

}  // namespace pmrc
