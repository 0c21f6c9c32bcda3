"""FP64 CPU oracle for the collisionless Boltzmann moment step (arXiv:1210.5246).

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The CUDA product path in
``paper_1210_5246_gb300`` never imports it and shares no code with it.
"""
