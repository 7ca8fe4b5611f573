"""The FP64 CPU oracle and its independent checkers: test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline leg and the
reference arm) may import, call, link or run anything in this package
(__graft_entry__.build() compiles its C sources); the library has no CPU
implementation of the path and never falls back to this one.
"""
