#pragma once
#include <cuda_runtime.h>

namespace jfnk {
bool prof_on();
// name: kernel class; work: elements processed by one launch
void prof_begin(const char* name, double work, cudaStream_t st);
void prof_end(cudaStream_t st);
}  // namespace jfnk
