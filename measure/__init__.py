"""Measurement drivers beside bench.py: the paper's experiments re-run on the
library (kernel ablation, Stein-MAP-Seq vs PF-MAP-Seq, scenario C latency)
and the learned-proposal benchmark. They call the library only through its
public binding; nothing here is imported by the library itself."""
