"""CPU oracle for the inverse p-th root iteration. Test infrastructure: imported only by tests/,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg."""
