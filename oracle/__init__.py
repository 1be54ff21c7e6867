"""FP64 CPU oracle for the Maxwell–Bloch FDTD step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import anything under this package.  The product
package ``paper_0809_1547_gb300`` never imports it, and the two share no code:
only the seeded input generators (``paper_0809_1547_gb300.inputs``, which hold
none of the method's arithmetic) feed both.
"""
