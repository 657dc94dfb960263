"""CPU oracle for the emulated ZGEMM and the KKR tau_00 solve -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import, call, link or execute anything in this
package.  The product path (``paper_2603_29975_gb300``) never touches it and shares no
code with it; the two meet only through the seeded inputs of ``synth``.

Modules
-------
ozaki    : Ozaki-I emulated complex GEMM written out step by step (numpy + Python ints).
kkr      : tau_00 = [(I - tG)^-1]_00 t_0 by full Gauss-Jordan inversion and by block LU.
mlp      : the slice-count selector network, forward and backward in numpy.
c_oracle : ctypes loader of the plain C oracle (``oracle/c/ozk_oracle.c``) used for the
           larger cases and for the timed CPU baseline.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against values
the mathematics fixes (see each docstring); the learned selector's *output* is
"parity unpinned" (it is a trained model) while its gradients are pinned.
"""
