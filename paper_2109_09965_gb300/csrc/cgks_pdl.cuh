// Programmatic dependent launch (sm_90 and later).
//
// The kernels of a cycle run back to back on one stream.  Launched with the
// programmatic-serialization attribute, kernel k+1 may be scheduled while
// kernel k is still running: its blocks become resident and wait in
// griddepcontrol.wait until kernel k has completed and its writes are
// visible, which hides the launch and block-scheduling latency of every
// kernel boundary.  Each kernel calls pdl_enter() before it touches data
// that a kernel of the cycle writes: the wait orders it after its
// predecessor (reads and writes alike).  Every thread waits, so a kernel
// completes only after its predecessor has, and the chain orders each
// kernel after all earlier ones.  Before the wait a kernel may read only
// mesh data, which nothing writes while cycles run.  pdl_exit() at the
// end of the kernel body lets the next kernel launch (blocks that return
// early count as done); where the trigger falls affects only timing, since
// the next kernel waits for this one to complete whatever happens.
// Launched without the attribute, the wait returns at once and the kernel
// is stream-ordered as usual.
#pragma once

namespace cgks {

// wait for the predecessor kernel (its writes visible)
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// let the next kernel be scheduled (at the end of the kernel body: an
// earlier trigger let the next grid take SM resources from this one and
// measured slower on GB300)
__device__ __forceinline__ void pdl_exit() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace cgks
