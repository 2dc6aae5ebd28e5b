__kernel void sysvals(__global uint *out)
{
    out[get_global_id(0)] = ((get_global_size(0) >> 1) ^ (((get_global_size(0) >> 4) & 15u) + (get_global_size(0) + (get_work_dim() * get_num_groups(1)))));
}
