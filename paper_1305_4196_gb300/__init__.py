"""GB300-native short-range molecular dynamics hot path (arXiv:1305.4196).

Submodules:
  workloads - seeded synthetic inputs (no method arithmetic)
  build     - nvcc build of libmdgb.so (sm_103a)
  mdgb      - Python binding of the C ABI (loads libmdgb.so; raises if it is missing)
  batch     - ensembles of independent systems (include/mdgb_batch.h)
  autograd  - torch.autograd.Function for force-matching derivatives
  waves     - the paper's wave schedule (host tool)
"""
