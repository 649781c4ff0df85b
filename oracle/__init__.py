"""CPU oracle for the complex CCSD iteration and its triples corrections (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import this package. It shares
no code with the CUDA library and never imports it.
"""
