"""TensorMD energy/force/virial hot path for GB300 (sm_103a)."""
