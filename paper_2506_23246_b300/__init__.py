"""B300-native QPINN hot path: batched statevector simulation of the paper's PQC
with exact input derivatives, Maxwell/energy losses and adjoint gradients.

The compute path is the C-ABI library ``libqpinn.so`` (hand-written sm_103a
CUDA). ``paper_2506_23246_b300.qp`` is its thin ctypes binding; importing this
package does not load the library, so the seeded workload generators in
``workloads`` can be used on machines without the extension.
"""
__all__ = ["qp", "workloads"]
