"""Plain CPU oracle of the GateKeeper-GPU filter (arxiv 2103.14978).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
"""
