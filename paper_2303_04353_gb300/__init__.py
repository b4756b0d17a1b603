"""Cascading double-double GEMM (Parikh, van de Geijn, Henry, arXiv
2303.04353) as hand-written sm_103a CUDA kernels behind a C ABI.

``_lib`` is the ctypes binding of include/ddgemm.h; ``ops`` wraps it for
PyTorch CUDA tensors (device memory and streams only).  Importing this
package loads nothing; the first call loads (and if needed builds) the
library and raises if it cannot."""
