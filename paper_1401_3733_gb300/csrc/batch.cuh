// batch.cuh -- the persistent multi-lattice launch of batch.cu as a building
// block: the even-odd normal operator Dhat^+ Dhat of several lattices (each
// with its own FP32 multi-RHS fields) in one cooperative launch.
#pragma once

#include "bsm_internal.cuh"

namespace bsm {

struct BatchNormalItem {
  bsm_lattice lat;  // SU(2) or SU(3) fundamental
  const void* U32;  // FP32 links
  const void* p;    // even multi-RHS half spinor (input)
  void* u;          // even: Dhat p
  void* t;          // odd temporary
  void* Mp;         // even: Dhat^+ Dhat p
  int nrhs;
};

// bytes of the control block the launch keeps at the start of its workspace
size_t batch_control_bytes();
// enqueues the launch on s (capturable); the barrier waits give up after
// timeout_s and set the error flag that batch_status reads
int batch_normal_launch(const BatchNormalItem* items, int count, void* ctl_ws, double timeout_s, cudaStream_t s);
// waits for s and reads the error flag: BSM_OK or BSM_ETIMEOUT
int batch_status(void* ws, cudaStream_t s);

}  // namespace bsm
